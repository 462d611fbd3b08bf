"""Factorize-and-solve with the forward sweep folded into the factorization
launch (stiles_factorize_solve) against the separate calls: the same factor
(bit for bit: the extra tasks only read it), the same log-determinant, and the
solution within FP64 rounding of stiles_solve's (the forward products are summed
in another order) and of the oracle's solve, with a small residual."""
import numpy as np
import pytest
import torch

from oracle import analyze as oan
from oracle import cholesky as och
from paper_2501_02483_b300 import build, inputs
from paper_2501_02483_b300 import stiles as st

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build_library()
    st.lib()


def _residual(m, x, b):
    A = inputs.dense_from_csc(m)
    return np.linalg.norm(A @ x - b, axis=0).max() / np.linalg.norm(b, axis=0).max()


@pytest.mark.parametrize("case", [
    dict(n=3000, arrow=24, hw=40, T=16, order=st.ORDER_ND, nrhs=4),
    dict(n=2999, arrow=7, hw=70, T=16, order=st.ORDER_RCM, nrhs=1),
    dict(n=2500, arrow=30, hw=90, T=32, order=st.ORDER_ND, nrhs=16),
    dict(n=2100, arrow=64, hw=120, T=64, order=st.ORDER_AUTO, nrhs=5),
    dict(n=1000, arrow=0, hw=30, T=16, order=st.ORDER_NONE, nrhs=3),
])
def test_fused_matches_separate_calls(case):
    m = inputs.band_arrow(case["n"], case["arrow"], case["hw"], 0.4, 11, nrhs=case["nrhs"])
    plan = st.Plan.from_matrix(m, tile=case["T"], ordering=case["order"])
    vd = torch.from_numpy(m["values"]).cuda()
    b = torch.from_numpy(np.asfortranarray(m["rhs"])).cuda()
    f1 = st.Factor(plan)
    f1.factorize(vd)
    x1 = f1.solve(b).cpu().numpy()
    f2 = st.Factor(plan)
    x2 = f2.factorize_solve(vd, b).cpu().numpy()
    assert np.array_equal(f1.tiles(), f2.tiles())
    assert f1.logdet() == f2.logdet()
    assert np.max(np.abs(x2 - x1)) <= 1e-12 * np.max(np.abs(x1))
    assert _residual(m, x2, m["rhs"]) <= 1e-12
    # element-wise against the oracle's solve of the same ordering and tile size
    p = oan.analyze(m, case["T"], case["order"])
    L = och.factorize(m, p["perm"], case["T"], p["tcolptr"], p["trowidx"])
    x_ref = och.solve(L, p["perm"], case["T"], p["tcolptr"], p["trowidx"], m["rhs"])
    assert np.max(np.abs(x2 - x_ref)) <= 1e-10 * np.max(np.abs(x_ref))
    # the factor it leaves solves like any other
    x3 = f2.solve(b).cpu().numpy()
    assert np.array_equal(x3, x1)


def test_fused_repeated_calls_reuse_the_factor():
    m = inputs.band_arrow(2000, 10, 50, 0.3, 3, nrhs=2)
    plan = st.Plan.from_matrix(m, tile=16, ordering=st.ORDER_ND)
    vd = torch.from_numpy(m["values"]).cuda()
    b = torch.from_numpy(np.asfortranarray(m["rhs"])).cuda()
    f = st.Factor(plan)
    xa = f.factorize_solve(vd, b).cpu().numpy()
    xb = f.factorize_solve(vd, b).cpu().numpy()
    assert np.array_equal(xa, xb)


def test_fused_not_spd_and_bad_arguments():
    d = np.ones(600)
    d[200] = -1.0
    m = inputs.diagonal_matrix(d)
    plan = st.Plan.from_matrix(m, tile=16, ordering=st.ORDER_NONE)
    b = torch.ones(600, 2, dtype=torch.float64).cuda().t().contiguous().t()
    with pytest.raises(st.StilesError) as e:
        st.Factor(plan).factorize_solve(torch.from_numpy(m["values"]).cuda(), b)
    assert e.value.name == "NOT_SPD" and e.value.info == 201
    # more right-hand sides than the block holds
    m2 = inputs.band_arrow(500, 4, 20, 0.3, 1)
    plan2 = st.Plan.from_matrix(m2, tile=16)
    bb = torch.ones(m2["n"], 17, dtype=torch.float64).cuda().t().contiguous().t()
    with pytest.raises(st.StilesError) as e2:
        st.Factor(plan2).factorize_solve(torch.from_numpy(m2["values"]).cuda(), bb)
    assert e2.value.name == "INVALID"
    # mixed-precision plans keep the separate calls
    plan3 = st.Plan.from_matrix(m2, tile=64, precision=st.PREC_F16)
    with pytest.raises(st.StilesError) as e3:
        st.Factor(plan3).factorize_solve(torch.from_numpy(m2["values"]).cuda(),
                                         torch.ones(m2["n"], dtype=torch.float64).cuda())
    assert e3.value.name == "UNSUPPORTED"


def test_fused_in_place_single_block_and_pure_arrowhead():
    """x may equal b; a matrix of one padded block; a pure arrowhead (diagonal
    body, dense arrow): the same results as the separate calls."""
    cases = [inputs.band_arrow(7, 3, 2, 0.5, 5, nrhs=1)]  # n = 10: one block of 16, padded
    pa = inputs.pure_arrowhead(400, 12, 3)
    pa = pa[0] if isinstance(pa, tuple) else pa
    cases.append(dict(pa, rhs=np.asfortranarray(np.random.default_rng(1).normal(size=(pa["n"], 3)))))
    for m in cases:
        plan = st.Plan.from_matrix(m, tile=16, ordering=st.ORDER_AUTO)
        vd = torch.from_numpy(m["values"]).cuda()
        b = torch.from_numpy(np.asfortranarray(m["rhs"])).cuda()
        f1 = st.Factor(plan)
        f1.factorize(vd)
        x1 = f1.solve(b).cpu().numpy()
        xb = b.clone()  # solved in place: x is b
        st.Factor(plan).factorize_solve(vd, xb, x=xb)
        x2 = xb.cpu().numpy()
        assert np.max(np.abs(x2 - x1)) <= 1e-12 * np.max(np.abs(x1))
        assert _residual(m, x2, m["rhs"]) <= 1e-12
