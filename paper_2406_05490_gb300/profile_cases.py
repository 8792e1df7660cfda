"""Small fixed workloads for profiling single kernels (e.g. under ncu): a few RK3 steps of one
configuration through the C ABI, nothing else.

    python -m paper_2406_05490_gb300.profile_cases low 2048 3      # low order, 2048^2, 3 steps
    python -m paper_2406_05490_gb300.profile_cases lowdf 2048 3    # the same in double words
    python -m paper_2406_05490_gb300.profile_cases high32 256 2     # FP32C high order
    python -m paper_2406_05490_gb300.profile_cases high64 128 2     # FP64 high order
    python -m paper_2406_05490_gb300.profile_cases batch 64 2       # 64 ragged interfaces
    python -m paper_2406_05490_gb300.profile_cases single 32 10     # single mode, free edges, FP64
"""
from __future__ import annotations

import sys


def main(argv):
    if len(argv) < 3:
        print(__doc__)
        return 2
    kind, size, steps = argv[0], int(argv[1]), int(argv[2])
    import torch

    from . import inputs, zm
    torch.cuda.set_device(0)
    if kind == "batch":
        insts = inputs.ragged_batch(count=size, lo=64, hi=384, n_modes=4, seed=0)
        h = zm.zm_batch_create([(r.n, r.n, 1.0, 1.0, True) for r in insts], [r.atwood for r in insts],
                               delta=[0.1 / r.n for r in insts])
        for k, r in enumerate(insts):
            zm.zm_batch_set_state(h, k, r.z, inputs.random_state(r.n, seed=k)[1])
        zm.zm_batch_step(h, 1e-3, steps)
        zm.zm_batch_sync(h)
        zm.zm_batch_destroy(h)
        return 0
    if kind == "single":
        z, w = inputs.single_mode(size)
        model = zm.ZModel(size, periodic=False, atwood=0.5, g=1.0, delta=0.1 / size)
        model.set_state(z, w)
        model.step(1e-3, steps)
        model.sync()
        model.close()
        return 0
    order = zm.ZM_ORDER_LOW if kind in ("low", "lowdf") else zm.ZM_ORDER_HIGH
    z, _ = inputs.multi_mode(size, n_modes=8, seed=7, amp=0.02)
    _, w = inputs.random_state(size, seed=3)
    model = zm.ZModel(size, periodic=True, atwood=0.7, g=1.0, order=order, fp32c=(kind == "high32"),
                      df64=(kind == "lowdf"))
    model.set_state(z, w)
    model.step(1e-3, steps)
    model.sync()
    model.close()
    return 0


if __name__ == "__main__":
    sys.exit(main(sys.argv[1:]))
