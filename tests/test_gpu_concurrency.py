"""An operator built on one stream by a second host thread while another
operator is solved on a second stream gives bit-identical tables and
solutions to the same work done one call at a time (the pipelined steps of
the bench rely on this)."""
import threading

import numpy as np
import pytest
import torch

from workloads import icosphere

pytestmark = pytest.mark.gpu

gb = pytest.importorskip("paper_2201_12050_gb300")

COUNTS, LATTICE = (6, 5, 1), np.diag([0.5, 0.55, 1.0])
KS = [2.0, 3.0, 4.5]


def _solve(op):
    b = op.rhs_plane_wave([[0.6, 0.8, 0.0]])
    p, info = op.solve(b, tol=1e-10, restart=80)
    return p.cpu(), info[0]["iters"]


def test_build_during_solve_matches_sequential_results():
    v, t = icosphere(1, 0.2)
    x = torch.ones((1, len(t) * 30), dtype=torch.complex128, device="cuda")
    ref = []
    for k in KS:
        op = gb.Operator(v, t, COUNTS, LATTICE, k, form=gb.FORM_PBEM)
        ref.append((op.matvec(x).cpu(), *_solve(op)))
        op.close()
    solve_stream = torch.cuda.Stream(priority=-1)
    build_stream = torch.cuda.Stream()
    built = {}

    def build(i):
        with torch.cuda.stream(build_stream):
            built[i] = gb.Operator(v, t, COUNTS, LATTICE, KS[i], form=gb.FORM_PBEM)

    th = threading.Thread(target=build, args=(0,))
    th.start()
    th.join()
    got = []
    for i in range(len(KS)):
        op = built.pop(i)
        th = None
        if i + 1 < len(KS):
            th = threading.Thread(target=build, args=(i + 1,))
            th.start()
        with torch.cuda.stream(solve_stream):
            y = op.matvec(x).cpu()
            p, iters = _solve(op)
        if th is not None:
            th.join()
        got.append((y, p, iters))
        op.close()
    for (y0, p0, it0), (y1, p1, it1) in zip(ref, got):
        assert torch.equal(y0, y1)
        assert torch.equal(p0, p1) and it0 == it1
