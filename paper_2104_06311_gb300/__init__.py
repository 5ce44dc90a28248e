"""GB300 (sm_103a) dual-polarisation coherent-receiver DSP chain.

The CUDA kernels live in ``csrc/`` and build into ``librx.so``
(``python -m paper_2104_06311_gb300.build``); ``rx`` is the ctypes binding of
the C ABI declared in ``include/rx.h`` (``Receiver``), ``include/rx_batch.h``
(``Batch``), ``include/rx_cnn.h`` (``CNN``), ``include/rx_kk.h`` (``KKFrontEnd``),
``include/rx_wl.h`` (``WLEqualiser``) and ``include/rx_rt.h`` (``RealTime``).
"""
from .rx import CNN, Batch, KKFrontEnd, RealTime, Receiver, WLEqualiser, load, q_db, RxError  # noqa: F401
