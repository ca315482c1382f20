"""The allocation-free batched entry point, called through the C ABI.

Some callers cannot allocate device memory at the point where they evaluate
PDFs: a host framework that reserved the whole device memory up front, or a
Monte Carlo event loop that must never trigger cudaMalloc (which can fail on a
full device and can synchronise the whole device).  `pdf_batch_run_noalloc`
runs the batched kernel with its scratch (tile ticket, request and grid
tables) in a fixed static device array instead.  This test checks it against
the regular prepared batch (`pdf_batch_prepare` + `pdf_batch_run`) on two
calls in a row -- bit for bit, since both launch the same kernel arithmetic
-- and against the oracle on a sample, that those calls leave the device's
free memory and torch's allocator untouched, and that it refuses requests
beyond its fixed capacity.

This file is collected last on purpose: it must pass alone in a fresh process
and after every other test.
"""
import ctypes as C

import numpy as np
import pytest

from oracle.oracle import OracleGrid
from paper_2012_08221_gb300 import synth
from tests import parity

pytestmark = pytest.mark.gpu
torch = pytest.importorskip("torch")


def _descs(reqs):
    from paper_2012_08221_gb300._lib import BatchDesc
    arr = (BatchDesc * len(reqs))()
    for i, (pdf, member, pids, x, q2, out) in enumerate(reqs):
        arr[i].grid = pdf.handle
        arr[i].member = int(member)
        arr[i].n_pid = int(pids.size)
        for k in range(pids.size):
            arr[i].pids[k] = int(pids[k])
        arr[i].x = x.data_ptr()
        arr[i].q2 = q2.data_ptr()
        arr[i].n = x.numel()
        arr[i].out = out.data_ptr()
    return arr


def test_noalloc_batch_matches_prepared_batch_twice():
    from paper_2012_08221_gb300 import build
    from paper_2012_08221_gb300._lib import lib
    from paper_2012_08221_gb300.batch import Batch
    from paper_2012_08221_gb300.pdf import PDF
    build.build()
    grids = [synth.grid_set_a(n_rep=7), synth.grid_set_b(), synth.grid_set_c(n_rep=5)]
    pdfs = [PDF.from_grid(g) for g in grids]
    batches = synth.batches_uneven(grids, n_batches=120, scale=0.01, seed=77)
    dev = torch.device("cuda")
    ref_reqs, new_reqs = [], []
    for b in batches:
        x = torch.as_tensor(b.x, device=dev)
        q2 = torch.as_tensor(b.q2, device=dev)
        shape = (b.x.size, b.pids.size)
        ref_reqs.append((pdfs[b.set_index], b.member, b.pids, x, q2,
                         torch.empty(shape, dtype=torch.float64, device=dev)))
        new_reqs.append((pdfs[b.set_index], b.member, b.pids, x, q2,
                         torch.empty(shape, dtype=torch.float64, device=dev)))
    B = Batch(ref_reqs, autotune=False)
    B.run()
    torch.cuda.synchronize()
    arr = _descs(new_reqs)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    # one call first, so that lazily loaded kernels and the array's address
    # lookup are behind us before the memory is measured
    assert lib().pdf_batch_run_noalloc(arr, len(new_reqs), stream) == 0, lib().pdf_last_error()
    torch.cuda.synchronize()
    for call in range(2):
        for r in new_reqs:
            r[5].fill_(float("nan") if call == 0 else -1.0)
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        stats0 = torch.cuda.memory_stats()
        rc = lib().pdf_batch_run_noalloc(arr, len(new_reqs), stream)
        assert rc == 0, lib().pdf_last_error()
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        stats1 = torch.cuda.memory_stats()
        assert free1 == free0, (free0, free1)
        for key in ("allocation.all.allocated", "segment.all.allocated", "allocated_bytes.all.allocated"):
            assert stats1.get(key, 0) == stats0.get(key, 0), key
        for r_ref, r_new in zip(ref_reqs, new_reqs):
            assert torch.equal(r_new[5], r_ref[5]), f"no-alloc call {call}"
    # and against the oracle on the first points of every tenth request
    orcs = [OracleGrid.from_synth(g) for g in grids]
    for b, r in list(zip(batches, new_reqs))[::10]:
        m = min(b.x.size, 500)
        o = orcs[b.set_index]
        want = o.xfxq2_batch(b.pids, b.x[:m], b.q2[:m], member=b.member)
        kap = o.kappa(b.pids, b.x[:m], b.q2[:m], member=b.member)
        parity.check(r[5][:m].cpu().numpy(), want, kap, what="no-alloc vs oracle")


def test_noalloc_after_a_narrower_prepared_batch():
    """A prepared batch of the same kernel shape whose output rows are
    narrower (1 pid) must leave the no-alloc launch (3 pids, more shared
    memory) free to run, in either order."""
    from paper_2012_08221_gb300 import build
    from paper_2012_08221_gb300._lib import lib
    from paper_2012_08221_gb300.batch import Batch
    from paper_2012_08221_gb300.pdf import PDF
    build.build()
    g = synth.grid_nnpdf()
    pdf = PDF.from_grid(g)
    dev = torch.device("cuda")
    x, q2, _ = synth.queries_nnpdf(70_001, seed=91)
    X, Q = torch.as_tensor(x, device=dev), torch.as_tensor(q2, device=dev)
    one = np.array([21], dtype=np.int32)
    three = np.array([-2, 21, 2], dtype=np.int32)
    narrow = [(pdf, 0, one, X, Q, torch.empty((x.size, 1), dtype=torch.float64, device=dev))]
    wide = [(pdf, 0, three, X, Q, torch.empty((x.size, 3), dtype=torch.float64, device=dev))]
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    B = Batch(narrow, autotune=False)
    for _ in range(2):
        B.run()
        rc = lib().pdf_batch_run_noalloc(_descs(wide), 1, stream)
        assert rc == 0, lib().pdf_last_error()
        torch.cuda.synchronize()
        assert torch.equal(wide[0][5], pdf.xfxQ2(three, X, Q))
        assert torch.equal(narrow[0][5], pdf.xfxQ2(one, X, Q))


def test_noalloc_batch_rejects_more_requests_than_its_capacity():
    from paper_2012_08221_gb300 import build
    from paper_2012_08221_gb300._lib import BatchDesc, lib
    build.build()
    arr = (BatchDesc * 1025)()
    rc = lib().pdf_batch_run_noalloc(arr, 1025, None)
    assert rc == -6                                   # PDF_E_RANGE
    assert b"1 to 1024 requests" in lib().pdf_last_error()


def test_noalloc_many_requests_span_several_parameter_blocks():
    """1000 requests (more than one copy kernel's worth of the request
    table; some of them empty) over three grids, bit for bit against the
    prepared batch."""
    from paper_2012_08221_gb300 import build
    from paper_2012_08221_gb300._lib import lib
    from paper_2012_08221_gb300.batch import Batch
    from paper_2012_08221_gb300.pdf import PDF
    build.build()
    grids = [synth.grid_set_a(n_rep=3), synth.grid_set_b(), synth.grid_set_c(n_rep=2)]
    pdfs = [PDF.from_grid(g) for g in grids]
    rng = np.random.default_rng(78)
    dev = torch.device("cuda")
    ref_reqs, new_reqs = [], []
    for i in range(1000):
        s = int(rng.integers(0, 3))
        g = grids[s]
        n = int(rng.integers(0, 300)) if i % 7 else 0
        x, q2, _ = synth.queries_nnpdf(max(n, 1), seed=5000 + i)
        x, q2 = x[:n], q2[:n]
        pids = rng.choice(g.pids, int(rng.integers(1, 4)), replace=False).astype(np.int32)
        member = int(rng.integers(0, g.n_members))
        X, Q = torch.as_tensor(x, device=dev), torch.as_tensor(q2, device=dev)
        for reqs in (ref_reqs, new_reqs):
            reqs.append((pdfs[s], member, pids, X, Q, torch.full((n, pids.size), -7.0, dtype=torch.float64,
                                                                 device=dev)))
    Batch(ref_reqs, autotune=False).run()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        rc = lib().pdf_batch_run_noalloc(_descs(new_reqs), len(new_reqs), stream)
        assert rc == 0, lib().pdf_last_error()
        torch.cuda.synchronize()
        for a, b in zip(ref_reqs, new_reqs):
            assert torch.equal(a[5], b[5])
