"""Small runs of every kernel family through the C ABI, for comparing the checked build
(libzm_checked.so: every kernel tests the indices it computes and counts violations) with the
default build.

    ZM_LIB=checked python tests/checked_cases.py OUT.npz

writes the outputs of each case and the checked build's violation count to OUT.npz.  Run by
tests/test_gpu_checked.py once per build; not collected by pytest itself.
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(out_path):
    import torch

    from paper_2406_05490_gb300 import inputs, zm

    torch.cuda.set_device(0)
    zm.load()
    zm.zm_bounds_status(clear=True)
    res = {}

    def model_case(name, n1, n2, periodic, order, fp32c=False, df64=False, mu=0.0, steps=2, cutoff=0.0):
        z, w = inputs.random_state(n1, n2, seed=n1 + 7 * n2, periodic=periodic)
        delta = 0.1 / max(n1, n2)
        m = zm.ZModel(n1, n2, periodic=periodic, atwood=0.6, g=1.2, mu=mu, delta=delta, order=order,
                      fp32c=fp32c, df64=df64)
        if cutoff:
            zm.zm_set_cutoff(m.h, cutoff)
        u, wd = m.velocity(z, w)
        m.set_state(z, w)
        m.step(1e-3, steps)
        zs, ws = m.get_state()
        m.close()
        res[name + "_u"], res[name + "_wd"], res[name + "_z"], res[name + "_w"] = u, wd, zs, ws

    H, LO, MED = zm.ZM_ORDER_HIGH, zm.ZM_ORDER_LOW, zm.ZM_ORDER_MEDIUM
    model_case("fp64_free", 32, 24, False, H)
    model_case("fp64_per", 40, 48, True, H, mu=0.01)
    model_case("fp32c", 64, 64, True, H, fp32c=True)
    model_case("fp32c_aniso", 32, 128, True, H, fp32c=True)
    model_case("fp32c_cut", 64, 64, True, H, fp32c=True, cutoff=0.2)
    model_case("low_p2", 64, 32, True, LO, mu=0.01)
    model_case("low_mix", 24, 40, True, LO)
    model_case("low_mix19", 608, 152, True, LO, steps=1)
    model_case("med64", 24, 40, True, MED)
    model_case("med32c", 32, 64, True, MED, fp32c=True)
    model_case("df_p2", 64, 32, True, LO, df64=True, mu=0.01)
    model_case("df_mix", 24, 40, True, LO, df64=True)
    model_case("df_mix19", 608, 152, True, LO, df64=True, steps=1)
    model_case("df_herm", 2048, 32, True, LO, df64=True, steps=1)

    # a ragged batch
    specs = [(37, 53, False), (64, 64, True), (5, 9, False), (48, 40, True)]
    h = zm.zm_batch_create([(a, b, 1.0, 1.0, p) for a, b, p in specs], [0.5] * len(specs), g=1.1,
                           delta=[0.1 / max(a, b) for a, b, _ in specs])
    for k, (a, b, p) in enumerate(specs):
        zm.zm_batch_set_state(h, k, *inputs.random_state(a, b, seed=k, periodic=p))
    zm.zm_batch_step(h, 1e-3, 2)
    zm.zm_batch_sync(h)
    # every other tile shape, one evaluation each (timing-based tuning would differ between runs)
    for tp1, tp2 in ((8, 32), (32, 8), (4, 64), (64, 4)):
        zm.zm_batch_set_tile_shape(h, tp1, tp2)
        zm.zm_batch_velocity(h)
        for k, (a, b, _) in enumerate(specs):
            ub = np.empty((3, a * b))
            zm.zm_batch_get_velocity(h, k, ub, None)
            res[f"batch{k}_u_{tp1}x{tp2}"] = ub
    for k, (a, b, _) in enumerate(specs):
        zb, wb = np.empty((3, a * b)), np.empty((2, a * b))
        zm.zm_batch_get_state(h, k, zb, wb)
        res[f"batch{k}_z"], res[f"batch{k}_w"] = zb, wb
    zm.zm_batch_destroy(h)

    # the serving loop on three small requests
    sv = zm.zm_server_create(1 << 28, 8)
    ids = []
    for k, n in enumerate((16, 24, 32)):
        z, w = inputs.random_state(n, seed=40 + k)
        ids.append((zm.zm_server_submit(sv, n, n, z, w, 0.5, 0.1 / n, 1e-3, 3), n))
    for rid, n in ids:
        zm.zm_server_wait(sv, rid, 60.0)
        st, zr, wr, _, _ = zm.zm_server_result(sv, rid, n * n)
        res[f"serve{n}_z"], res[f"serve{n}_w"] = zr, wr
        res[f"serve{n}_status"] = np.array([st])
    zm.zm_server_destroy(sv)

    # the allocation-free FP64 sum on caller buffers
    n = 300
    z, w = inputs.random_state(20, 15, seed=3)
    zt = torch.from_numpy(z[:, :n].copy()).cuda()
    gt = torch.from_numpy(np.vstack([w, w[:1]])[:, :n].copy()).cuda()
    ut = torch.empty((3, n), dtype=torch.float64, device="cuda")
    zm.zm_br_velocity_noalloc(n, zt, gt, 0.01, ut)
    torch.cuda.synchronize()
    res["noalloc_u"] = ut.cpu().numpy()

    hits, first, line = zm.zm_bounds_status(clear=True)
    res["checked"] = np.array([int(zm.zm_checked_build())])
    res["hits"] = np.array([hits, first, line], dtype=np.int64)
    np.savez(out_path, **res)
    print(f"checked={int(zm.zm_checked_build())} hits={hits} first={first} line={line} cases={len(res)}")


if __name__ == "__main__":
    main(sys.argv[1])
