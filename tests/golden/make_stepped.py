"""Write the oracle's stepped states of the full-size high-order configurations.

The stored arrays are computed by the CPU oracle alone (oracle/, built with OpenMP: the
Birkhoff-Rott sums split their targets across threads and return the same bits as the serial
build) from the seeded inputs of paper_2406_05490_gb300.inputs; nothing here touches the GPU
library.  The GPU tests step the same initial states through the C ABI and compare.

    python tests/golden/make_stepped.py            # both cases (about 10 minutes on 8 cores)
    python tests/golden/make_stepped.py 256        # only the 256^2 case

Cases (periodic unit square, g = 1, mu = 0, delta = 0.1 dx, dt = 1e-3, SSP-RK3, high order):
  multimode256_20: 256^2, z3 = 16 modes, (kx, ky) in [2, 8], amplitudes N(0, 0.01), phases
                   U[0, 2 pi) from seed 0, w = 0, A = 0.5, 20 steps (the 256^2 multi-mode run).
  multimode512_1:  512^2, z3 = 8 modes of amplitude 0.02 from seed 7, w = 0, A = 0.7, 1 step
                   (the high-order half of the low-order vs high-order comparison).
Each file holds z3_0 (the initial heights, so that the GPU test starts from the very same bits),
the final z (3, N) and w (2, N), and a JSON description with the oracle source's SHA-256.
"""
from __future__ import annotations

import hashlib
import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

CASES = {
    "multimode256_20": dict(n=256, n_modes=16, seed=0, amp=None, atwood=0.5, steps=20),
    "multimode512_1": dict(n=512, n_modes=8, seed=7, amp=0.02, atwood=0.7, steps=1),
}


def oracle_source_sha256():
    h = hashlib.sha256()
    for name in ("zm_oracle.c", "zm_oracle.h"):
        h.update(open(os.path.join(ROOT, "oracle", name), "rb").read())
    return h.hexdigest()


def path_of(name):
    return os.path.join(HERE, f"stepped_{name}.npz")


def initial_state(case):
    from paper_2406_05490_gb300 import inputs
    kw = {} if case["amp"] is None else {"amp": case["amp"]}
    return inputs.multi_mode(case["n"], n_modes=case["n_modes"], seed=case["seed"], **kw)


def write(name):
    import oracle
    case = CASES[name]
    n = case["n"]
    z0, w0 = initial_state(case)
    m = oracle.Mesh(n, periodic=True)
    t0 = time.time()
    z, w = oracle.run(m, z0, w0, case["atwood"], 1.0, 0.0, 0.1 / n, 1e-3, case["steps"])
    secs = time.time() - t0
    meta = dict(case, name=name, g=1.0, mu=0.0, delta=0.1 / n, dt=1e-3, order="high",
                periodic=True, oracle_sha256=oracle_source_sha256(), oracle_seconds=round(secs, 1),
                threads=os.environ.get("OMP_NUM_THREADS", str(os.cpu_count())))
    np.savez_compressed(path_of(name), z3_0=z0[2], z=z, w=w, meta=np.array(json.dumps(meta)))
    print(f"{name}: {secs:.0f} s -> {path_of(name)}")


def main(argv):
    import oracle
    # the OpenMP build of the same oracle source (same bits as the serial build)
    os.environ["ZM_ORACLE_LIB"] = oracle.build(openmp=True)
    names = [k for k in CASES if not argv or any(a in k for a in argv)]
    for name in names:
        write(name)
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
