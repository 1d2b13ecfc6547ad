"""Run by tests/test_gpu_debug_build.py in a child process: the same sampling calls under the
library it loads (SAIS_DEBUG=1 selects the debug build), results written to an .npz file."""
import sys

import numpy as np
import torch

from paper_2501_04971_gb300 import sais, workloads as wl


def batch():
    return [wl.qkp(100, 0.5, 1), wl.qkp(600, 0.5, 2), wl.qkp(1000, 0.25, 3, profit_max=10000),
            wl.mkp(60, 12, 4), wl.qkp(300, 0.75, 5)]


def main(out_path):
    torch.cuda.set_device(0)
    res = {}
    insts = batch()
    prob = sais.Problem(insts)
    lam = torch.full((prob.count * prob.m_stride,), 0.7, device="cuda:0")
    for variant, k in (("plain", 0), ("auto", 0)):
        out = prob.sample(lam, 160, 12, 10.0, 3, 1, variant=variant, block_k=k)
        prob.synchronize()
        for key, v in out.items():
            res[f"{variant}_{key}"] = v.cpu().numpy()
    prob.set_auto_mode("groups")
    out = prob.sample(lam, 160, 12, 10.0, 3, 1, variant="auto")
    prob.synchronize()
    res["groups_x"] = out["x"].cpu().numpy()
    r = prob.solve(3, 128, 10, 10.0, 20.0, 9, variant="auto", use_graph=True)
    res["solve_best_cost"] = r["best_cost"]
    prob.close()
    # the rank-k kernels (resident, streamed) and the block-field kernel at K = 32
    for insts2, k in (([wl.qkp(200, 0.5, 6), wl.qkp(400, 0.5, 7)], 16),
                      ([wl.qkp(300, 0.5, 8)], 32)):
        p2 = sais.Problem(insts2)
        lam2 = torch.full((p2.count * p2.m_stride,), 0.7, device="cuda:0")
        out = p2.sample(lam2, 128, 10, 10.0, 3, 0, variant="blocked", block_k=k)
        p2.synchronize()
        res[f"blocked{k}_x"] = out["x"].cpu().numpy()
        p2.close()
    # the reporting path: a check that fails by construction (debug build) or is refused
    p3 = sais.Problem([wl.qkp(40, 0.5, 9)])
    try:
        p3.debug_check_selftest()
        try:
            p3.synchronize()
            res["selftest"] = np.array([0])
        except sais.SaisError as e:
            res["selftest"] = np.array([e.status])
            res["selftest_msg"] = np.array([str(e)])
        p3.synchronize()   # the status words were reset
    except sais.SaisError as e:
        res["selftest"] = np.array([-e.status])
    p3.close()
    np.savez(out_path, **res)


if __name__ == "__main__":
    main(sys.argv[1])
