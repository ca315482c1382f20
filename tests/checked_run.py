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
        out[extrap] = {"status": p.status(), "digest": digest(*[r for r in res if r.dtype == torch.float64])}
    vg = Vegas(3, n_bins=20)
    r, jac, bins = vg.map(torch.rand((20_000, 3), dtype=torch.float64, device=dev))
    vg.accumulate(jac, bins)
    print(json.dumps(out))
    return 0


if __name__ == "__main__":
    sys.exit(main())
