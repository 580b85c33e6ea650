"""Batched persistent launch: every problem of a batch must equal the same
problem advanced alone through hard_hydro_advance (same kernel arithmetic,
bit for bit), and sampled problems must match the FP64 oracle."""
import numpy as np
import pytest

import hydro_inputs as H
import oracle

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu
hh = pytest.importorskip("paper_2509_08971_gb300")


def small_spec(nprob, seed):
    # the batched configuration's recipe with sizes cut down for the tests
    return H.batch_spec(nprob, seed=seed, n1d=(16, 700), n2d=(8, 70))


@pytest.mark.parametrize("dtype", [torch.float32, torch.float64])
@pytest.mark.parametrize("tile", [0, 1, 2])
def test_batch_equals_problems_run_alone(dtype, tile):
    spec = small_spec(40, seed=tile)
    B = hh.HardBatch(spec.nx, spec.ny, spec.gamma, hh.HARD_BC_OUTFLOW, dtype=dtype, tile=tile)
    states = [H.batch_problem_U(spec, q) for q in range(spec.nprob)]
    packed = B.pack(states)
    t = B.step(packed, 12, 0.4)
    assert B.get_error() == hh.HARD_OK
    tb = t.cpu().numpy()
    for q in range(spec.nprob):
        m = hh.HardHydro((1, int(spec.ny[q]), int(spec.nx[q])), float(spec.gamma[q]),
                         hh.HARD_BC_OUTFLOW, dtype=dtype)
        U = torch.tensor(states[q], dtype=dtype, device="cuda")
        t1, _, _ = m.advance(U, 12, 0.4)
        assert torch.equal(B.view(packed, q), U), q
        assert float(t1) == tb[q], q


def test_batch_matches_oracle_fp64():
    spec = small_spec(12, seed=7)
    B = hh.HardBatch(spec.nx, spec.ny, spec.gamma, hh.HARD_BC_OUTFLOW, dtype=torch.float64)
    states = [H.batch_problem_U(spec, q) for q in range(spec.nprob)]
    packed = B.pack(states)
    t = B.step(packed, 8, 0.4).cpu().numpy()
    for q in range(spec.nprob):
        g = oracle.Grid((1, int(spec.ny[q]), int(spec.nx[q])), float(spec.gamma[q]),
                        oracle.BC_OUTFLOW)
        ref, t_ref, _ = g.run(states[q], 8, 0.4)
        got = B.view(packed, q).double().cpu().numpy()
        scale = np.max(np.abs(ref.reshape(5, -1)), axis=1) + 1e-300
        err = np.max(np.abs(got - ref).reshape(5, -1), axis=1) / scale
        assert np.all(err <= 1e-12), (q, err)
        assert t[q] == pytest.approx(t_ref, rel=1e-14)


def test_batch_graph_replay_and_uneven_sizes():
    """One captured graph replayed twice equals two direct calls; a batch mixes
    1D problems of 2 cells up to 2D problems of several tiles."""
    nx = [2, 3, 700, 64, 33, 100, 17]
    ny = [1, 1, 1, 64, 33, 9, 40]
    gam = [1.4, 1.67, 1.3, 1.4, 1.4, 1.5, 1.4]
    B = hh.HardBatch(nx, ny, gam, hh.HARD_BC_PERIODIC)
    rng = np.random.default_rng(3)
    states = []
    for q in range(len(nx)):
        W = [rng.uniform(0.5, 2.0, (1, ny[q], nx[q])), rng.uniform(-0.5, 0.5, (1, ny[q], nx[q])),
             rng.uniform(-0.5, 0.5, (1, ny[q], nx[q])), np.zeros((1, ny[q], nx[q])),
             rng.uniform(0.5, 2.0, (1, ny[q], nx[q]))]
        states.append(H.prim_to_cons(W, gam[q]))
    direct = B.pack(states)
    td = B.step(direct, 5, 0.3)
    B.step(direct, 5, 0.3, t=td)
    replayed = B.pack(states)
    tr = torch.zeros(len(nx), dtype=torch.float64, device="cuda")
    g = B.capture(replayed, 5, 0.3, tr)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(direct, replayed)
    assert torch.equal(td, tr)


def test_batch_rejects_bad_problems_and_flags_nonphysical():
    assert hh.hard_batch_create(2, [1, 8], [1, 1], [1, 1], [1.4, 1.4], [1, 1], 0) is None
    assert hh.hard_batch_create(1, [8], [8], [2], [1.4], [1], 0) is None
    assert hh.hard_batch_create(1, [8], [8], [1], [0.9], [1], 0) is None
    B = hh.HardBatch([16, 8], [1, 8], 1.4)
    U = [H.prim_to_cons([np.ones((1, 1, 16)), np.zeros((1, 1, 16)), np.zeros((1, 1, 16)),
                         np.zeros((1, 1, 16)), np.ones((1, 1, 16))], 1.4),
         H.prim_to_cons([np.ones((1, 8, 8)), np.zeros((1, 8, 8)), np.zeros((1, 8, 8)),
                         np.zeros((1, 8, 8)), np.ones((1, 8, 8))], 1.4)]
    U[1][0, 0, 3, 3] = -1.0
    packed = B.pack(U)
    B.step(packed, 1, 0.4)
    assert B.get_error() == hh.HARD_ENONPHYS
