"""FP64 CPU oracle of the coherent-receiver DSP chain.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, obviously correct
statement of what the receiver computes, used to check the CUDA library.  Only
the tests, ``__graft_entry__.smoke()`` and the CPU-baseline / reference legs of
``bench.py`` may import it.  The product path (``paper_2104_06311_gb300``) never
imports, links or executes anything here, and this package shares no code with
it.

Every function cites the passage of the paper (arXiv 2104.06311) it is the
analogue of.  Steps on which the paper is silent (CMA, the butterfly MIMO,
blind phase search, the frequency-offset estimator, LLRs, the dispersion
transfer function) follow the textbook definitions written out in
``oracle.chain``'s docstrings.

Parity status: every function in ``oracle.chain`` is pinned by a
``-m "not gpu"`` test in ``tests/test_oracle_pins.py`` (closed forms,
invariants, brute force, BER theory); ``oracle.cnn`` by
``tests/test_cnn_pins.py``; the Kramers-Kronig front end ``oracle.kk`` by
``tests/test_kk_pins.py`` (exact reconstruction of a minimum-phase field,
identity overlap-save, decimation, the carrier's dispersion phase, stream
continuity); the widely-linear DD-LMS ``oracle.wl`` by ``tests/test_wl_pins.py``
(fixed point, zero-step convolution, closed-form IQ-imbalance inverse, schedule
locality, AWGN BER).  None is marked "parity unpinned".
"""
from .chain import (  # noqa: F401
    RxParams, n_cd_taps, default_overlap, default_fft_n, cd_response, rrc_response,
    cdc_filter, cdc_overlap_save, bps_outer_angles, region_bounds, lms_step,
    decide, hard_bits, llr_maxlog, fo_estimate_sum, ring_weight, equalize, bps_outer, demap,
    run_chain, ber_sync_count, q_from_ber, ber_theory,
)
