"""GPU checks of the batched factorization (one persistent launch over many
matrices, Appendix A) and of the tile-size autotuner.

* every matrix of a batch gets the oracle's log-determinant and a solve with a
  1e-12 (FP64) / 1e-10 (refined BF16) residual;
* each factor in the mix is bitwise identical to the same matrix factorized
  alone (the task graph and the arithmetic per task do not depend on the
  batch);
* a non-SPD matrix is reported per matrix with the oracle's column, the others
  still succeed;
* replaying the batch with new values (a hyperparameter sweep) is correct.
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


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build_library()
    st.lib()


def _mats(count, seed):
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        nb = int(rng.integers(300, 3000))
        out.append(inputs.band_arrow(nb, int(rng.integers(0, 30)), int(rng.choice([8, 24, 60])), 0.3,
                                     int(rng.integers(0, 1 << 30)), nrhs=2))
    return out


@pytest.mark.parametrize("prec,T,order", [(st.PREC_F64, 16, st.ORDER_NONE), (st.PREC_F64, 32, st.ORDER_ND),
                                          (st.PREC_BF16, 64, st.ORDER_NONE), (st.PREC_SLICED, 32, st.ORDER_ND)])
def test_batch_matches_oracle_and_single(prec, T, order):
    mats = _mats(9, 7 + T)
    plans = [st.Plan.from_matrix(m, tile=T, ordering=order, precision=prec) for m in mats]
    batch = st.Batch(plans)
    vals = [torch.from_numpy(m["values"]).cuda() for m in mats]
    statuses, infos = batch.factorize(vals)
    assert np.all(statuses == 0)
    lds = batch.logdets()
    tol_ld = {st.PREC_F64: 1e-12, st.PREC_SLICED: 1e-8}.get(prec, 1e-7)
    tol_rr = 1e-12 if prec == st.PREC_F64 else 1e-10
    for i, m in enumerate(mats):
        p = oan.analyze(m, T, order)
        Lo = och.factorize(m, p["perm"], T, p["tcolptr"], p["trowidx"])
        ld_o = och.logdet(Lo, p["nt"])
        v = batch.factor(i)
        assert abs(lds[i] - ld_o) <= tol_ld * abs(ld_o)
        assert abs(v.logdet() - lds[i]) <= 1e-13 * abs(lds[i])
        x, rr = v.solve(m["rhs"], relres=True)
        assert rr <= tol_rr
        # alone vs in the mix: the same bits
        f = st.Factor(plans[i])
        f.factorize(vals[i])
        assert np.array_equal(f.tiles(), v.tiles())
    batch.close()


def test_batch_reports_non_spd_per_matrix():
    mats = _mats(5, 3)
    bad = 2
    vals = mats[bad]["values"].copy()
    vals[mats[bad]["colptr"][100]] = -5.0  # a negative diagonal entry in column 100
    mats[bad] = dict(mats[bad], values=vals)
    plans = [st.Plan.from_matrix(m, tile=16, ordering=st.ORDER_NONE) for m in mats]
    batch = st.Batch(plans)
    statuses, infos = batch.factorize([m["values"] for m in mats], raise_on_error=False)
    with pytest.raises(och.NotSPD) as eo:
        p = oan.analyze(mats[bad], 16, oan.ORDER_NONE)
        och.factorize(mats[bad], p["perm"], 16, p["tcolptr"], p["trowidx"])
    assert statuses[bad] == 2 and infos[bad] == eo.value.info
    assert np.all(np.delete(statuses, bad) == 0)
    batch.close()


def test_batch_replay_with_new_values_theta_sweep():
    mats = _mats(6, 11)
    plans = [st.Plan.from_matrix(m, tile=16) for m in mats]
    batch = st.Batch(plans)
    batch.factorize([m["values"] for m in mats])
    ld1 = batch.logdets()
    thetas = np.linspace(0.5, 2.0, len(mats))
    batch.factorize([m["values"] * t for m, t in zip(mats, thetas)])
    ld2 = batch.logdets()
    for m, t, a, b in zip(mats, thetas, ld1, ld2):
        assert abs(b - (a + m["n"] * math.log(t))) <= 1e-12 * abs(b)
    batch.close()


def test_autotune_picks_a_candidate():
    m = inputs.band_arrow(20000, 20, 100, 0.3, 1)
    best, ms = st.autotune(m, [16, 32, 64, 512])
    assert best in (16, 32, 64, 512)
    assert ms[[16, 32, 64, 512].index(best)] == min(t for t in ms if t > 0)
    assert ms[3] == -1.0 or ms[3] >= min(t for t in ms if t > 0)


@pytest.mark.parametrize("prec,T,order", [(st.PREC_F64, 16, st.ORDER_NONE), (st.PREC_F64, 32, st.ORDER_ND),
                                          (st.PREC_BF16, 64, st.ORDER_NONE), (st.PREC_F16, 64, st.ORDER_ND)])
def test_batch_solve_matches_single_and_oracle(prec, T, order):
    """One forward + one backward launch over the whole batch: every matrix's x
    meets the residual bound against its own A; FP64 solutions are bitwise the
    single-matrix solve's (same task lists, same arithmetic); mixed-precision
    matrices refine independently; mixed right-hand-side counts, a skipped
    matrix, host and device right-hand sides."""
    mats = _mats(11, 101 + T)
    plans = [st.Plan.from_matrix(m, tile=T, ordering=order, precision=prec) for m in mats]
    batch = st.Batch(plans)
    vals = [torch.from_numpy(m["values"]).cuda() for m in mats]
    statuses, _ = batch.factorize(vals)
    assert np.all(statuses == 0)
    rng = np.random.default_rng(T)
    rhs = []
    for i, m in enumerate(mats):
        k = [1, 3, 16, 7, 0][i % 5]
        if k == 0:
            rhs.append(None)
            continue
        b = np.asfortranarray(rng.standard_normal((m["n"], k)))
        rhs.append(torch.from_numpy(b).cuda() if i % 2 else b)
    xs, rel, its, status = batch.solve(rhs)
    assert status == 0
    tol = 1e-12 if prec == st.PREC_F64 else 1e-10
    for i, m in enumerate(mats):
        if rhs[i] is None:
            assert xs[i] is None and rel[i] == 0.0
            continue
        b = rhs[i] if isinstance(rhs[i], np.ndarray) else rhs[i].cpu().numpy()
        x = xs[i] if isinstance(xs[i], np.ndarray) else xs[i].cpu().numpy()
        assert isinstance(xs[i], np.ndarray) == isinstance(rhs[i], np.ndarray)
        A = inputs.dense_from_csc(m)
        rr = np.linalg.norm(b - A @ x, axis=0) / np.linalg.norm(b, axis=0)
        assert rr.max() <= tol * 10, (i, rr.max())
        assert rel[i] <= tol
        xs1 = batch.factor(i).solve(b)
        if prec == st.PREC_F64:
            assert its[i] == 0
            assert np.array_equal(x, xs1)
        else:
            assert its[i] >= 1
            assert np.max(np.abs(x - xs1)) <= 1e-8 * np.max(np.abs(x))
    batch.close()


@pytest.mark.parametrize("prec,T", [(st.PREC_BF16, 64), (st.PREC_SLICED, 32)])
def test_batch_residual_every_rhs_count(prec, T):
    """Matrix i of the batch solves i + 1 right-hand sides (1 .. 16): the batched
    residual product runs one instantiation per count, and refinement stops on
    it, so the reported relres of every matrix must match ||b - A x|| / ||b||
    formed on the host from the dense A."""
    rng = np.random.default_rng(5)
    mats = [inputs.band_arrow(int(rng.integers(300, 1500)), int(rng.integers(0, 20)), int(rng.choice([8, 24, 60])),
                              0.3, int(rng.integers(0, 1 << 30))) for _ in range(16)]
    plans = [st.Plan.from_matrix(m, tile=T, ordering=st.ORDER_ND, precision=prec) for m in mats]
    batch = st.Batch(plans)
    statuses, _ = batch.factorize([torch.from_numpy(m["values"]).cuda() for m in mats])
    assert np.all(statuses == 0)
    rhs = [np.asfortranarray(rng.standard_normal((m["n"], i + 1))) for i, m in enumerate(mats)]
    xs, rel, its, status = batch.solve(rhs)
    assert status == 0
    for i, m in enumerate(mats):
        assert xs[i].shape == rhs[i].shape
        A = inputs.dense_from_csc(m)
        rr = np.linalg.norm(rhs[i] - A @ xs[i], axis=0) / np.linalg.norm(rhs[i], axis=0)
        assert rr.max() <= 1e-10, (i, rr.max())
        assert abs(rel[i] - rr.max()) <= 0.05 * rr.max() + 1e-14, (i, rel[i], rr.max())
    batch.close()


def test_batch_solve_oracle_solution_small():
    """The batched solve against the oracle's own triangular solves on C0-sized
    matrices (independent of the single-matrix path)."""
    mats = _mats(4, 55)
    plans = [st.Plan.from_matrix(m, tile=16, ordering=st.ORDER_RCM) for m in mats]
    batch = st.Batch(plans)
    batch.factorize([m["values"] for m in mats])
    xs, rel, _, _ = batch.solve([m["rhs"] for m in mats])
    for i, m in enumerate(mats):
        p = oan.analyze(m, 16, oan.ORDER_RCM)
        Lo = och.factorize(m, p["perm"], 16, p["tcolptr"], p["trowidx"])
        xo = och.solve(Lo, p["perm"], 16, p["tcolptr"], p["trowidx"], m["rhs"])
        assert np.max(np.abs(xs[i] - xo)) <= 1e-10 * np.max(np.abs(xo))
    batch.close()


def test_batch_solve_rejects_bad_counts():
    mats = _mats(2, 9)
    plans = [st.Plan.from_matrix(m, tile=16) for m in mats]
    batch = st.Batch(plans)
    batch.factorize([m["values"] for m in mats])
    with pytest.raises(st.StilesError):
        batch.solve([np.zeros((mats[0]["n"], 17)), None])
    batch.close()
