"""LHAPDF "lhagrid1" sets: read through the library's native reader, and a
writer for grids made here (PDFFlow Sec. 1 and 4 keep this community format).

``read_set(folder, first_member, n_members)`` returns a grid object the PDF
class accepts; ``load(folder, ...)`` builds the PDF on the GPU directly;
``write_set(folder, grid)`` writes a grid (e.g. a synthetic one) as a set.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import synth
from ._lib import GridDesc, check, lib


def read_set(folder: str, first_member: int = 0, n_members: int = 1) -> synth.Grid:
    """Members [first_member, first_member + n_members) as host arrays (no GPU)."""
    h = C.c_void_p()
    check("pdf_lhapdf_open", lib().pdf_lhapdf_open(os.fsencode(folder), first_member, n_members, C.byref(h)))
    try:
        d = GridDesc()
        check("pdf_lhapdf_desc", lib().pdf_lhapdf_desc(h, C.byref(d)))
        nx, ns, nf, nm = d.n_x, d.n_sub, d.n_flav, d.n_members
        x = np.ctypeslib.as_array(d.x_knots, shape=(nx,)).copy()
        nq = np.ctypeslib.as_array(d.n_q, shape=(ns,)).copy()
        rows = int(nq.sum())
        q = np.ctypeslib.as_array(d.q_knots, shape=(rows,)).copy()
        pids = np.ctypeslib.as_array(d.pids, shape=(nf,)).copy()
        v = np.ctypeslib.as_array(d.values, shape=(nm, rows, nx, nf)).copy()
        a = np.ctypeslib.as_array(d.alphas, shape=(rows,)).copy() if d.alphas else None
    finally:
        lib().pdf_lhapdf_close(h)
    return synth.Grid(x, nq, q, pids, v, a, os.path.basename(os.path.normpath(folder)))


def load(folder: str, first_member: int = 0, n_members: int = 1, device="cuda:0", **kw):
    """A PDF object for the set's members (``mkPDF("set/member")`` of the paper)."""
    from .pdf import PDF
    return PDF.from_grid(read_set(folder, first_member, n_members), device=device, **kw)


def write_set(folder: str, grid, set_desc: str = "synthetic grid") -> None:
    """Write ``grid`` (all its members) as an lhagrid1 set in ``folder``."""
    name = os.path.basename(os.path.normpath(folder))
    os.makedirs(folder, exist_ok=True)
    pids = [21 if int(p) == 0 else int(p) for p in grid.pids]
    qk = np.asarray(grid.q_knots)
    info = [f'SetDesc: "{set_desc}"', "Format: lhagrid1", "DataVersion: 1",
            f"NumMembers: {grid.n_members}", f"Flavors: [{', '.join(str(p) for p in pids)}]",
            "Interpolator: logbicubic", "Extrapolator: continuation",
            f"XMin: {grid.x_knots[0]:.17e}", f"XMax: {grid.x_knots[-1]:.17e}",
            f"QMin: {qk[0]:.17e}", f"QMax: {qk[-1]:.17e}"]
    if grid.alphas is not None:
        info.append("AlphaS_Qs: [" + ", ".join(f"{v:.17e}" for v in qk) + "]")
        info.append("AlphaS_Vals: [" + ", ".join(f"{v:.17e}" for v in grid.alphas) + "]")
    with open(os.path.join(folder, name + ".info"), "w") as f:
        f.write("\n".join(info) + "\n")
    starts = np.concatenate([[0], np.cumsum(grid.n_q)])
    for m in range(grid.n_members):
        lines = [f"PdfType: {'central' if m == 0 else 'replica'}", "Format: lhagrid1", "---"]
        for s in range(len(grid.n_q)):
            r0, r1 = starts[s], starts[s + 1]
            lines.append(" ".join(f"{v:.17e}" for v in grid.x_knots))
            lines.append(" ".join(f"{v:.17e}" for v in qk[r0:r1]))
            lines.append(" ".join(str(p) for p in pids))
            for ix in range(grid.n_x):
                for r in range(r0, r1):
                    lines.append(" ".join(f"{v:.17e}" for v in grid.values[m, r, ix]))
            lines.append("---")
        with open(os.path.join(folder, f"{name}_{m:04d}.dat"), "w") as f:
            f.write("\n".join(lines) + "\n")
