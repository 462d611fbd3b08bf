"""GPU checks of the continuous-batching request loop.

* every request of a Poisson stream completes with a refined residual <= 1e-10;
* each served result equals the same request served alone (factor, logdet and
  solution: the batched launch computes bit-identical factors, the solution
  agrees to the refinement tolerance);
* re-solves use resident factors; with a tiny HBM budget factors are evicted,
  misses are counted and refactorized, and the answers stay correct;
* jobs overlap on the device: per-job CUDA events (and the persistent
  kernels' own events) on one device clock show two jobs in flight at once,
  and every result of that run still equals the request served alone.
"""
import numpy as np
import pytest

from paper_2501_02483_b300 import build, inputs
from paper_2501_02483_b300 import serve as sv
from paper_2501_02483_b300 import stiles as st

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


@pytest.fixture(scope="module", autouse=True)
def built():
    build.build_library()
    st.lib()


def _stream(count, seed):
    specs, arrivals = inputs.serving_workload(count, rate=2000.0, seed=seed, n_lo=500, n_hi=8000, hw_hi=96,
                                              w_hi=20, nrhs_hi=4, pool=6)
    return [sv.Request(d["id"], d["kind"], d["key"], d["matrix"], d["rhs"], d["target"]) for d in specs], arrivals


def _check_alone(reqs, prec, tile):
    by_id = {r.id: r for r in reqs}
    for r in reqs:
        assert r.status == 0 and r.relres <= 1e-10
        src = r if r.kind == "new" else by_id[r.target]
        plan = st.Plan.from_matrix(src.matrix, tile=tile, precision=prec)
        f = st.Factor(plan)
        f.factorize(src.matrix["values"])
        assert f.logdet() == pytest.approx(r.logdet, rel=1e-13)
        x = f.solve(r.rhs)
        assert np.max(np.abs(x - r.x)) <= 1e-9 * np.max(np.abs(x))


@pytest.mark.parametrize("prec", [st.PREC_BF16, st.PREC_F64, st.PREC_SLICED])
def test_served_results_equal_alone(prec):
    reqs, arrivals = _stream(30, 1)
    tile = {st.PREC_F64: 16, st.PREC_SLICED: 32}.get(prec, 64)
    srv = sv.Server(precision=prec, tile=tile, max_batch=8)
    done = srv.run(reqs, arrivals)
    assert len(done) == len(reqs)
    assert srv.stats["batches"] >= 2  # later arrivals were admitted into later launches
    _check_alone(reqs, prec, tile)
    srv.close()


def test_jobs_overlap_on_the_device_and_results_equal_alone():
    """Two workers: jobs overlap on the device (per-job events), and so do the
    persistent factorization kernels of two jobs.  Whether two kernels meet in a
    given run depends on when each worker's host-side set-up ends, so the run is
    repeated (up to three times) until they do; every run's results must equal
    the requests served alone."""
    kernel_overlap = []
    for attempt in range(3):
        reqs, arrivals = _stream(40, 3 + attempt)
        srv = sv.Server(precision=st.PREC_F64, tile=16, max_batch=4, gpu_workers=2)
        done = srv.run(reqs, arrivals)
        assert len(done) == len(reqs)
        both, busy, peak = srv.overlap()
        assert peak >= 2 and both > 0, (both, busy, peak)
        kboth, kbusy, kpeak = srv.overlap(kernels=True)
        kernel_overlap.append((kboth, kbusy, kpeak))
        # the job intervals lie inside the run and every factor job has a kernel window
        iv = srv.intervals()
        assert all(0.0 <= a < b for _, a, b, _ in iv)
        assert len(srv.kernels) == sum(1 for k, *_ in iv if k == "factor")
        _check_alone(reqs, st.PREC_F64, 16)
        srv.close()
        if kpeak >= 2 and kboth > 0:
            break
    assert any(kp >= 2 and kb > 0 for kb, _, kp in kernel_overlap), kernel_overlap


def test_eviction_refactorizes_and_stays_correct():
    reqs, arrivals = _stream(24, 2)
    srv = sv.Server(precision=st.PREC_BF16, tile=64, max_batch=4, hbm_budget=5e6)
    done = srv.run(reqs, arrivals)
    assert len(done) == len(reqs)
    assert srv.stats["evicted_batches"] > 0
    for r in reqs:
        assert r.status == 0 and r.relres <= 1e-10
    srv.close()
