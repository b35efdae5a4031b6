"""Uneven member groups in one batch: handles of different grid sizes,
Reynolds numbers, horizons and ensemble sizes advance together, one captured CUDA graph per chunk.
Every handle runs the same kernels on the same data as in its own forward run, so costs, gradients
and states must agree bit for bit with the separate runs, and the first of them with the oracle."""
import numpy as np
import pytest

import oracle
import paper_2605_23812_gb300 as pkg
from paper_2605_23812_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    import __graft_entry__
    __graft_entry__.build()


# (nx, ny, Re, n_steps, N): horizons in the ratio 1 : 2 : 4 of the uneven configuration
GROUPS = [(32, 16, 500.0, 40, 3), (64, 32, 1000.0, 80, 5), (128, 64, 2000.0, 160, 4)]


def make(nx, ny, Re, n, N, precision):
    cfg = pkg.default_config(nx, ny, Re=Re, n_steps=n, n_window=n // 2, n_members=N, precision=precision)
    ens = pkg.Ensemble(cfg)
    ens.set_initial_state(*synth.cavity_ic(nx, ny))
    return ens


@pytest.mark.parametrize("precision", [pkg.MIXED, pkg.FP64_BATCHED])
def test_batch_equals_separate_runs(precision):
    ws = [synth.weights(g[4], seed=10 + k) for k, g in enumerate(GROUPS)]
    sep = []
    for g, w in zip(GROUPS, ws):
        ens = make(*g, precision)
        ens.forward_ensemble(w)
        sep.append((ens.cost()[0], ens.gradient(), ens.get_state(g[4])[0].cpu().numpy()))
        ens.close()
    ens = [make(*g, precision) for g in GROUPS]
    batch = pkg.Batch(ens)
    n_chunks, per = batch.info()
    assert n_chunks == 4 and list(per) == [10, 20, 40]
    for _ in range(2):   # the second forward replays the captured chunk graph
        batch.forward(ws)
        for e, g, ref in zip(ens, GROUPS, sep):
            assert np.array_equal(e.cost()[0], ref[0])
            assert np.array_equal(e.gradient(), ref[1])
            assert np.array_equal(e.get_state(g[4])[0].cpu().numpy(), ref[2])
            assert (e.member_status() == 0).all()
    batch.close()
    for e in ens:
        e.close()
    if precision == pkg.FP64_BATCHED:
        nx, ny, Re, n, N = GROUPS[0]
        P = oracle.cavity_params(nx, ny, Re)
        u0, v0 = synth.cavity_ic(nx, ny)
        E = oracle.ensemble_seeded(P, 0.1, 0.05, N, 1000)
        ref = oracle.envar_gradient(P, u0, v0, E, ws[0], 1e-2, n, n // 2, nthreads=4)
        np.testing.assert_allclose(sep[0][0], ref["J"], rtol=1e-6)


def test_batch_rejects_plain_handles():
    e = make(32, 16, 500.0, 10, 2, pkg.FP64_PLAIN)
    with pytest.raises(pkg.EnvarError, match="EINVAL"):
        pkg.Batch([e])
    e.close()
