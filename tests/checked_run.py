"""Every form of the hot path on the range-checked library (run in a child
process with PDFGPU_CHECKED=1, since the library is chosen at import):
prints one JSON line with the status bits each form left and a digest of
its outputs, for comparison with the release library."""
import hashlib
import json
import math
import sys

import numpy as np
import torch

from paper_2012_08221_gb300 import build, synth


def digest(*tensors):
    h = hashlib.sha256()
    for t in tensors:
        h.update(np.ascontiguousarray(t.detach().cpu().numpy()).tobytes())
    return h.hexdigest()[:16]


def main():
    build.build()
    from paper_2012_08221_gb300.batch import Batch
    from paper_2012_08221_gb300.lumi import DeviceEvents, luminosity, luminosity_backward
    from paper_2012_08221_gb300.pdf import PDF
    from paper_2012_08221_gb300.vegas import Vegas, VegasLumi
    dev = torch.device("cuda")
    out = {"library": build.LIB}
    g = synth.grid_nnpdf(seeds=(1005, 1006))
    for extrap in ("linear", "freeze", "error", "continuation"):
        p = PDF.from_grid(g, extrap=extrap)
        x, q2, qa = synth.queries_nnpdf(100_003, seed=61)
        x[:50] = np.exp(np.linspace(math.log(1e-12), 0.0, 50))          # below and at the grid edges
        q2[:50] = np.exp(np.linspace(math.log(0.01), math.log(1e12), 50))
        X, Q, QA = (torch.as_tensor(a, device=dev) for a in (x, q2, qa))
        p.status()
        f = p.xfxQ2(g.pids, X, Q, member=1)
        a = p.alphasQ2(QA)
        pid = torch.as_tensor(np.random.default_rng(62).choice(g.pids, x.size).astype(np.int32), device=dev)
        fp = p.xfxQ2_pw(pid, X, Q)
        res = [f, a, fp]
        if extrap != "continuation":
            gv = torch.zeros(g.values.shape[1:], dtype=torch.float64, device=dev)
            gx, gq, _ = p.xfxQ2_backward(pid, X, Q, torch.ones(x.size, dtype=torch.float64, device=dev),
                                         pointwise=True, grad_values=gv)
            res += [gx, gq]
            # the same through the adjoint tape (its cells are range-checked too)
            T = p.new_tape(x.size)
            res += [p.xfxQ2_pw(pid, X, Q, tape=T), p.xfxQ2(g.pids, X, Q, member=1, tape=T)]
            gt = torch.zeros_like(gv)
            gxt, gqt, _ = p.xfxQ2_backward(pid, X, Q, torch.ones(x.size, dtype=torch.float64, device=dev),
                                           pointwise=True, grad_values=gt, tape=T)
            res += [gxt, gqt]
            # and with the derivative tape
            D = p.new_dtape(x.size)
            res.append(p.xfxQ2_pw(pid, X, Q, tape=T, dtape=D))
            gd = torch.zeros_like(gv)
            gxd, gqd, _ = p.xfxQ2_backward(pid, X, Q, torch.ones(x.size, dtype=torch.float64, device=dev),
                                           pointwise=True, grad_values=gd, tape=T, dtape=D)
            res += [D[:2 * x.size], D[2 * x.size:].view(torch.int32)[:x.size], gxd, gqd]
            # the matrix form's sorted adjoint (up to 16 columns)
            gm = torch.zeros_like(gv)
            pm = np.array([g.pids[0], 21, 9], dtype=np.int32)                  # 9: absent
            gxm, gqm, _ = p.xfxQ2_backward(pm, X, Q, torch.ones((x.size, 3), dtype=torch.float64, device=dev),
                                           member=1, grad_values=gm)
            res += [gxm, gqm]
        ev = DeviceEvents.from_host(synth.events_lhc(50_001, seed=63))
        L, lum, als = luminosity(p, ev)
        res += [lum, als]
        if extrap != "continuation":
            gl = torch.zeros(g.values.shape[1:], dtype=torch.float64, device=dev)
            luminosity_backward(p, ev, 1.0, gl)
        reqs = [(p, m, np.array(pp, dtype=np.int32), X[:n], Q[:n],
                 torch.empty((n, len(pp)), dtype=torch.float64, device=dev))
                for m, pp, n in ((0, [-1, 21], 70_001), (1, [5], 33_333), (0, [2, 3, -4], 1000))]
        Batch(reqs, autotune=False).run()
        res += [r[5] for r in reqs]
        u = torch.as_tensor(np.random.default_rng(64).uniform(0, 1, (40_000, 2)), device=dev)
        VegasLumi(p, math.log(1e-6), 2 * math.log(13000.0), n_bins=40).iteration(u)
        torch.cuda.synchronize()
        out[extrap] = {"status": p.status(),
                       "digest": digest(*[r for r in res if r.dtype in (torch.float64, torch.int32)])}
    vg = Vegas(3, n_bins=20)
    r, jac, bins = vg.map(torch.rand((20_000, 3), dtype=torch.float64, device=dev))
    vg.accumulate(jac, bins)
    # randomly shaped grids (2-knot subgrids, two x knots, x_max below 1...)
    from tests.tinygrids import random_grid
    for seed in range(12):
        gr, rng = random_grid(7000 + seed)
        p = PDF.from_grid(gr, interp=seed % 3, extrap=(seed // 3) % 4)
        U, W = np.log(gr.x_knots), np.log(gr.q_knots ** 2)
        x = np.exp(rng.uniform(U[0] - 3.0, 0.0, 20_001))
        q2 = np.exp(rng.uniform(W[0] - 3.0, W[-1] + 3.0, 20_001))
        X, Q = torch.as_tensor(x, device=dev), torch.as_tensor(q2, device=dev)
        p.status()
        res = [p.xfxQ2(gr.pids, X, Q), p.alphasQ2(Q)]
        pid = torch.as_tensor(rng.choice(gr.pids, x.size).astype(np.int32), device=dev)
        if (seed // 3) % 4 != 3:
            T = p.new_tape(x.size)
            res.append(p.xfxQ2_pw(pid, X, Q, tape=T))
            gv = torch.zeros(gr.values.shape[1:], dtype=torch.float64, device=dev)
            gx, gq, _ = p.xfxQ2_backward(pid, X, Q, torch.ones(x.size, dtype=torch.float64, device=dev),
                                         pointwise=True, grad_values=gv, tape=T)
            res += [gx, gq]
            gm = torch.zeros_like(gv)
            gxm, gqm, _ = p.xfxQ2_backward(gr.pids, X, Q,
                                           torch.ones((x.size, gr.pids.size), dtype=torch.float64, device=dev),
                                           grad_values=gm)
            res += [gxm, gqm]
            if gr.pids.size <= 16:
                ev = DeviceEvents.from_host(synth.events_lhc(5_001, seed=64 + seed))
                L, lum, als = luminosity(p, ev)
                res.append(lum)
                gl = torch.zeros(gr.values.shape[1:], dtype=torch.float64, device=dev)
                luminosity_backward(p, ev, 1.0, gl)
        bp = gr.pids[:2].copy()
        out2 = torch.empty((x.size, bp.size), dtype=torch.float64, device=dev)
        Batch([(p, 0, bp, X, Q, out2)], autotune=False).run()
        res.append(out2)
        torch.cuda.synchronize()
        out[f"random{seed}"] = {"status": p.status(), "digest": digest(*res)}
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
