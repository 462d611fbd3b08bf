"""GPU checks of the mixed-precision factorization (BF16 / FP16 tile updates on
tensor cores, FP32 accumulation and triangular solves, FP64 diagonal tiles and
FP64 iterative refinement of the solves).

Tolerances are stated per result against the FP64 oracle:
* factor entries: |L_lp - L| <= 4 u_lp max|L| (u_lp = 2^-8 for BF16, 2^-11 for
  FP16: the tile updates are products of rounded operands, accumulated in FP32);
* log-determinant: relative 1e-6 here; the measured error (~1e-9 on these
  inputs) is asserted below 1e-7 and reported by the benchmark;
* solves: ||b - A x|| / ||b|| <= 1e-10 after refinement (the stated target).
"""
import math

import numpy as np
import pytest

from oracle import analyze as oan
from oracle import cholesky as och
from paper_2501_02483_b300 import build, inputs
from paper_2501_02483_b300 import stiles as st

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)

ULP = {st.PREC_BF16: 2.0 ** -8, st.PREC_F16: 2.0 ** -11}


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build_library()
    st.lib()


def _check(m, T, order, prec, **kw):
    p = oan.analyze(m, T, order)
    Lo = och.factorize(m, p["perm"], T, p["tcolptr"], p["trowidx"])
    plan = st.Plan.from_matrix(m, tile=T, ordering=order, precision=prec, **kw)
    assert np.array_equal(plan.perm(), p["perm"])
    f = st.Factor(plan)
    f.factorize(torch.from_numpy(m["values"]).cuda())
    tiles = f.tiles()
    tc, tr = plan.tilemap()
    n = m["n"]
    worst, scale = 0.0, 0.0
    for k in range(tc.size - 1):
        for e in range(tc[k], tc[k + 1]):
            i = int(tr[e])
            g = tiles[e].T[:min(T, n - i * T), :min(T, n - k * T)]
            worst = max(worst, float(np.max(np.abs(g - Lo[(i, k)]))))
            scale = max(scale, float(np.max(np.abs(Lo[(i, k)]))))
    assert worst <= 4 * ULP[prec] * scale, worst / scale
    ld_o = och.logdet(Lo, p["nt"])
    ld = f.logdet()
    assert abs(ld - ld_o) <= 1e-7 * abs(ld_o), (ld, ld_o)
    b = m["rhs"] if m.get("rhs") is not None else np.random.default_rng(0).normal(size=(n, 2))
    x, rr = f.solve(b, relres=True)
    assert rr <= 1e-10
    xo = och.solve(Lo, p["perm"], T, p["tcolptr"], p["trowidx"], b)
    assert np.max(np.abs(x - xo)) <= 1e-8 * np.max(np.abs(xo))
    return plan, f


@pytest.mark.parametrize("prec", [st.PREC_BF16, st.PREC_F16])
def test_small_config_mixed(prec):
    _check(inputs.config_small(0), 64, oan.ORDER_NONE, prec)


@pytest.mark.parametrize("prec,order", [(st.PREC_BF16, oan.ORDER_ND), (st.PREC_F16, oan.ORDER_RCM)])
def test_ragged_multi_tile_mixed(prec, order):
    m = inputs.band_arrow(3001, 37, 90, 0.35, 5)
    _check(m, 64, order, prec)


@pytest.mark.parametrize("chunk,fanin", [(1, 2), (4, 16)])
def test_tree_shapes_mixed(chunk, fanin):
    m = inputs.band_arrow(2500, 70, 20, 0.5, 9)
    plan, f = _check(m, 64, oan.ORDER_NONE, st.PREC_BF16, tree_chunk=chunk, tree_fanin=fanin)
    assert plan.info()["nscratch"] > 0


def test_tile_128_runs_on_64_wide_subtiles():
    m = inputs.band_arrow(2000, 20, 100, 0.3, 4)
    plan, f = _check(m, 128, oan.ORDER_NONE, st.PREC_BF16)
    assert plan.info()["block"] == 64


def test_scaling_pin_mixed():
    m = inputs.config_small(0)
    theta = 0.7
    plans = [st.Plan.from_matrix(mm, tile=64, precision=st.PREC_BF16) for mm in (m, inputs.scaled(m, theta))]
    lds = []
    for plan, mm in zip(plans, (m, inputs.scaled(m, theta))):
        f = st.Factor(plan)
        f.factorize(mm["values"])
        lds.append(f.logdet())
    assert abs(lds[1] - (lds[0] + m["n"] * math.log(theta))) <= 1e-7 * abs(lds[1])


def test_not_spd_mixed():
    d = np.ones(500)
    d[321] = -3.0
    m = inputs.diagonal_matrix(d)
    plan = st.Plan.from_matrix(m, tile=64, precision=st.PREC_BF16)
    with pytest.raises(st.StilesError) as e:
        st.Factor(plan).factorize(m["values"])
    assert e.value.name == "NOT_SPD" and e.value.info == 322


def test_refinement_gives_up_with_not_converged():
    """Zero refinement budget and an unreachable tolerance: NOT_CONVERGED, x is
    still the refined-so-far iterate."""
    m = inputs.config_small(0)
    plan = st.Plan.from_matrix(m, tile=64, precision=st.PREC_BF16, refine_tol=1e-300, max_refine=1)
    f = st.Factor(plan)
    f.factorize(m["values"])
    with pytest.raises(st.StilesError) as e:
        f.solve(m["rhs"])
    assert e.value.name == "NOT_CONVERGED"


def test_stalled_refinement_switches_to_preconditioned_cg():
    """A BF16 factor of a matrix whose Schur complement is 1e-3 of its norm is too
    inaccurate for refinement to converge; the solve hands over to conjugate
    gradients preconditioned by that factor and still reaches refine_tol."""
    m = inputs.near_singular_arrowhead(3000, 40, 1e-3, 1)
    p = st.Plan.from_matrix(m, tile=64, precision=st.PREC_BF16)
    f = st.Factor(p)
    f.factorize(m["values"])
    x, rr = f.solve(m["rhs"], relres=True)
    assert rr <= 1e-10
    assert f.cg_iters() >= 1 and f.refine_iters() >= f.cg_iters()
    A = inputs.dense_from_csc(m)
    xo = np.linalg.solve(A, m["rhs"])
    assert np.max(np.abs(x - xo)) <= 1e-5 * np.max(np.abs(xo))
    # a well-conditioned one never leaves refinement
    m2 = inputs.near_singular_arrowhead(3000, 40, 1e-1, 2)
    p2 = st.Plan.from_matrix(m2, tile=64, precision=st.PREC_BF16)
    f2 = st.Factor(p2)
    f2.factorize(m2["values"])
    _, rr2 = f2.solve(m2["rhs"], relres=True)
    assert rr2 <= 1e-10 and f2.cg_iters() == 0


def test_in_place_device_solve_keeps_b_for_residuals():
    m = inputs.config_small()
    p = st.Plan.from_matrix(m, tile=64, precision=st.PREC_F16)
    f = st.Factor(p)
    f.factorize(m["values"])
    b = torch.from_numpy(np.asfortranarray(m["rhs"])).cuda()
    ref, _ = f.solve(b.clone(), relres=True)
    x, rr = f.solve(b, x=b, relres=True)
    assert rr <= 1e-10
    assert torch.allclose(x, ref, rtol=1e-9, atol=0)


@pytest.mark.parametrize("pos", [1, 17, 40, 63])
def test_not_spd_mixed_position_in_tile(pos):
    """The first bad pivot is reported at every depth of the 64 x 64 diagonal
    tile's blocked POTRF (16-wide leaves, 32- and 64-wide levels)."""
    d = np.ones(320)
    col = 128 + pos
    d[col] = -2.0
    d[col + 5] = -1.0  # a later bad pivot (same leaf, or the next tile) must not win
    m = inputs.diagonal_matrix(d)
    plan = st.Plan.from_matrix(m, tile=64, ordering=st.ORDER_NONE, precision=st.PREC_F16)
    with pytest.raises(st.StilesError) as e:
        st.Factor(plan).factorize(m["values"])
    assert e.value.name == "NOT_SPD" and e.value.info == col + 1


def test_mixed_diagonal_tiles_are_fp64_cholesky():
    """A block-diagonal matrix of dense 64 x 64 SPD blocks has no off-diagonal
    tiles, so its mixed-precision factor is the FP64 POTRF of each diagonal tile
    on the FP32-rounded input the mixed path stores: it must match numpy's FP64
    Cholesky of the same rounded blocks to FP64 accuracy (the 16-bit operand
    tolerance of the other mixed tests would hide an error here)."""
    rng = np.random.default_rng(7)
    nb = 5
    n = 64 * nb
    rows, cols, vals, blocks = [], [], [], []
    for b in range(nb):
        G = rng.standard_normal((64, 64))
        A = (G @ G.T / 64 + (0.05 + 0.5 * b) * np.eye(64)) * 10.0 ** (3 * (b - 2))
        blocks.append(A)
        i, j = np.tril_indices(64)
        rows.append(i + 64 * b)
        cols.append(j + 64 * b)
        vals.append(A[i, j])
    colptr, rowidx, values = inputs.coo_to_csc_lower(n, np.concatenate(rows), np.concatenate(cols),
                                                     np.concatenate(vals))
    m = {"n": n, "n_arrow": 0, "colptr": colptr, "rowidx": rowidx, "values": values, "rhs": None,
         "name": "blockdiag64"}
    plan = st.Plan.from_matrix(m, tile=64, ordering=st.ORDER_NONE, precision=st.PREC_F16)
    f = st.Factor(plan)
    f.factorize(values)
    tiles = f.tiles()
    tc, tr = plan.tilemap()
    assert np.array_equal(np.diff(tc), np.ones(nb, dtype=tc.dtype))  # diagonal tiles only
    for b in range(nb):
        L = tiles[tc[b]].T
        Lref = np.linalg.cholesky(blocks[b].astype(np.float32).astype(np.float64))
        # L is stored in FP32: compare within FP32 rounding of an FP64-accurate factor
        assert np.max(np.abs(L - Lref)) <= 2.0 ** -23 * np.max(np.abs(Lref))
        assert np.all(np.triu(L, 1) == 0.0)
    ld = f.logdet()
    ld_ref = sum(2.0 * np.log(np.diag(np.linalg.cholesky(A.astype(np.float32).astype(np.float64)))).sum()
                 for A in blocks)
    assert abs(ld - ld_ref) <= 1e-12 * abs(ld_ref)
