"""The batched form's CDC autotuner table persists across processes in the file
RX_TUNE_CACHE names, keyed by the GPU model: a fresh process writes this GPU's
entries (every FFT size with the radix-16 engine, N = 4096 also with the four-step
engine), and a second fresh process takes its FFT size and engine from the file
(planted values steer the choice) instead of measuring again; other GPUs' lines
stay, and a line without the engine field reads as engine 0."""
import json
import os
import subprocess
import sys

import pytest

from chain_helpers import ensure_built

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SNIPPET = """
import json, sys
sys.path.insert(0, {root!r})
from paper_2104_06311_gb300 import Batch
b = Batch([dict(baud=10e9, L_km=300.0, max_samples=1 << 16)])
print(json.dumps(dict(N=b.get_param(0, "FFT_N"), V=b.get_param(0, "OVERLAP"),
                      ns=b.get_param(0, "CDC_NS_PER_SAMPLE"), eng=b.get_param(0, "CDC_ENGINE"))))
"""


def _run(path):
    env = dict(os.environ, RX_TUNE_CACHE=path)
    r = subprocess.run([sys.executable, "-c", SNIPPET.format(root=ROOT)], env=env, capture_output=True, text=True,
                       timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_tuning_table_persists_per_gpu(tmp_path):
    ensure_built()
    path = str(tmp_path / "tune.txt")
    with open(path, "w") as f:
        f.write("Some Other GPU|99|1024|123.0\n")
    first = _run(path)
    lines = open(path).read().splitlines()
    assert "Some Other GPU|99|1024|123.0" in lines
    mine = [l for l in lines if not l.startswith("Some Other GPU")]
    assert len(mine) == 8                              # N = 256 .. 16384, and 4096 four-step
    key = mine[0].rsplit("|", 3)[0]
    assert sorted(tuple(map(int, l.rsplit("|", 3)[1:3])) for l in mine) == \
        sorted([(N, 0) for N in (256, 512, 1024, 2048, 4096, 8192, 16384)] + [(4096, 1)])
    # plant a table where N = 2048 is by far the cheapest per output sample (one line in
    # the format without the engine field)
    with open(path, "w") as f:
        f.write("Some Other GPU|99|1024|123.0\n")
        for N in (256, 512, 1024, 2048, 4096, 8192, 16384):
            f.write(f"{key}|{N}|0|{1.0 if N == 2048 else 1e6}\n" if N != 512 else f"{key}|{N}|1e6\n")
        f.write(f"{key}|4096|1|1e6\n")
    second = _run(path)
    assert second["N"] == 2048 and second["eng"] == 0, (first, second)
    assert abs(second["ns"] - 1.0 / (2048 - second["V"])) < 1e-9
    # the four-step engine at N = 4096 the cheapest
    with open(path, "w") as f:
        for N in (256, 512, 1024, 2048, 4096, 8192, 16384):
            f.write(f"{key}|{N}|0|1e6\n")
        f.write(f"{key}|4096|1|1.0\n")
    third = _run(path)
    assert third["N"] == 4096 and third["eng"] == 1, third
    assert len(open(path).read().splitlines()) == 8      # nothing measured again
    with open(path, "w") as f:
        f.write("Some Other GPU|99|1024|123.0\n")
    _run(path)
    assert open(path).read().splitlines()[0] == "Some Other GPU|99|1024|123.0"
