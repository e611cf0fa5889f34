"""The split-line stage kernels (Stage A over a slab, Stage B over the gathered slab pairs, Stage C
over a slab) against the oracle's Thomas solve of the whole lines: through the schedule on one
rank, and with W slabs of every line emulated in one process (the exchanges as the tensor moves
an all-to-all would make), for one and two right-hand sides and uneven slabs."""
import numpy as np
import pytest
import torch

import oracle as O
from parity import rel_err
import paper_2509_03933_gb300 as tdma
from paper_2509_03933_gb300.split_line import SlabStages, SplitLineSolver

pytestmark = pytest.mark.gpu


def _problem(n, L, nrhs, seed):
    rng = np.random.default_rng(seed)
    a = rng.uniform(-1, 0, (n, L))
    c = rng.uniform(-1, 0, (n, L))
    b = 2 + np.abs(a) + np.abs(c) + rng.uniform(0, 1, (n, L))
    d = rng.uniform(-1, 1, (n, L) + ((nrhs,) if nrhs > 1 else ()))
    return a, b, c, d


def _by_line(x):
    """[lines, n(, nrhs)] from a [n][lines(, nrhs)] array."""
    return np.swapaxes(np.asarray(x), 0, 1)


def _ref(a, b, c, d, nrhs):
    if nrhs == 1:
        return O.thomas(a.T, b.T, c.T, d.T).T
    return np.stack([O.thomas(a.T, b.T, c.T, d[..., q].T).T for q in range(nrhs)], axis=-1)


@pytest.mark.parametrize("n,L,batch", [(300, 1000, 256), (2, 50, 64), (64, 129, 7)])
def test_one_rank_through_the_schedule(n, L, batch):
    a, b, c, d = _problem(n, L, 1, n + L)
    t = [torch.from_numpy(v).cuda() for v in (a, b, c, d)]
    x = torch.zeros_like(t[3])
    st = SlabStages(n, L, (L, L, 1, 0), nrhs=1, first=True, last=True)
    SplitLineSolver(st, L, batch).solve(*t, x)
    assert st.last_error() == 0
    assert rel_err(_by_line(x.cpu().numpy()), _by_line(_ref(a, b, c, d, 1))) <= 1e-12


@pytest.mark.parametrize("W", [2, 4, 7])
@pytest.mark.parametrize("nrhs", [1, 2])
def test_slabs_emulated_in_one_process(W, nrhs):
    n, L = 97, 300
    a, b, c, d = _problem(n, L, nrhs, 10 * W + nrhs)
    A, B, C, D = (torch.from_numpy(v).cuda() for v in (a, b, c, d))
    X = torch.zeros_like(D)
    rows = [(n * r // W, n * (r + 1) // W) for r in range(W)]
    stages, scratch, red = [], [], []
    for r, (r0, r1) in enumerate(rows):  # Stage A on every "rank"
        st = SlabStages(r1 - r0, L, (L, L, 1, 0), nrhs=nrhs, first=r == 0, last=r == W - 1)
        sc = st.scratch(L)
        rd = torch.empty(L * st.K, dtype=torch.float64, device="cuda")
        st.reduce(A[r0:r1], B[r0:r1], C[r0:r1], D[r0:r1], 0, L, rd, sc)
        stages.append(st)
        scratch.append(sc)
        red.append(rd)
    gathered = torch.stack(red)  # [W][L][K]: what the owner of all lines gathers
    ends = torch.empty(W * L * stages[0].E, dtype=torch.float64, device="cuda")
    stages[0].pairs_solve(W, L, gathered, ends, stages[0].work(W, L))
    ends = ends.view(W, L * stages[0].E)
    for r, (r0, r1) in enumerate(rows):  # Stage C on every "rank" with its own end values
        stages[r].finish(0, L, ends[r].contiguous(), scratch[r], X[r0:r1])
    assert all(st.last_error() == 0 for st in stages)
    assert rel_err(_by_line(X.cpu().numpy()), _by_line(_ref(a, b, c, d, nrhs))) <= 1e-12


def test_singular_slab_sets_status():
    n, L = 16, 40
    a, b, c, d = _problem(n, L, 1, 3)
    a[:], c[:] = 0.0, 0.0
    b[5, 7] = 0.0  # line 7 is singular
    t = [torch.from_numpy(v).cuda() for v in (a, b, c, d)]
    x = torch.zeros_like(t[3])
    st = SlabStages(n, L, (L, L, 1, 0))
    SplitLineSolver(st, L, 16).solve(*t, x)
    assert st.last_error() == 5
    assert st.last_error() == 0


def test_batch_estimator_against_timing_every_candidate():
    # the paper's estimator (stage times measured once per candidate batch, pipeline modelled)
    # against timing the whole solve for every candidate, on one rank
    from paper_2509_03933_gb300.split_line import choose_batch
    n, L = 256, 65536
    a, b, c, d = _problem(n, L, 1, 77)
    t = [torch.from_numpy(v).cuda() for v in (a, b, c, d)]
    x = torch.zeros_like(t[3])
    st = SlabStages(n, L, (L, L, 1, 0))
    stage_times, measured = {}, {}
    for batch in (L, L // 4, L // 16):
        sol = SplitLineSolver(st, L, batch)
        stage_times[batch] = sol.measure_stages(*t, x)
        sol.solve(*t, x)  # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        sol.solve(*t, x)
        e1.record()
        e1.synchronize()
        measured[batch] = e0.elapsed_time(e1)
    best, est = choose_batch(L, stage_times)
    assert measured[best] <= 1.5 * min(measured.values())
    assert rel_err(_by_line(x.cpu().numpy()), _by_line(_ref(a, b, c, d, 1))) <= 1e-12


@pytest.mark.parametrize("m,first,last,nrhs", [(2, True, False, 1), (3, False, False, 2), (17, False, False, 1),
                                               (40, False, True, 1), (97, True, True, 2)])
def test_slab_reduce_records_match_the_stage_oracle(m, first, last, nrhs):
    # Stage A of one slab (the slab is one partition) against the oracle's modified-Thomas Stage A,
    # row by row: the reduced record (row 0 in x_{-1} and x_{m-1}, row m-1 in x_0 and x_m) and the
    # interior relations the slab keeps for Stage C (the forward form, alpha x_0 + x_t + gamma x_{t+1}
    # = delta), per line
    L = 300
    a, b, c, d = _problem(m, L, nrhs, 7 * m + nrhs)
    A, B, C, D = (torch.from_numpy(v).cuda() for v in (a, b, c, d))
    st = SlabStages(m, L, (L, L, 1, 0), nrhs=nrhs, first=first, last=last)
    sc = st.scratch(L)
    rd = torch.empty(L * st.K, dtype=torch.float64, device="cuda")
    st.reduce(A, B, C, D, 0, L, rd, sc)
    assert st.last_error() == 0
    al, cl = a.T.copy(), c.T.copy()
    if first:
        al[:, 0] = 0.0
    if last:
        cl[:, -1] = 0.0
    o = O.modified_thomas_partition(al, b.T, cl, np.swapaxes(d, 0, 1))
    de = o["delta"] if nrhs == 2 else o["delta"][..., None]
    want = np.concatenate([np.stack([o["alpha"][:, 0], o["gamma"][:, 0], o["alpha"][:, m - 1],
                                     o["gamma"][:, m - 1]], axis=1), de[:, 0, :], de[:, m - 1, :]], axis=1)
    rec = rd.view(L, st.K).cpu().numpy()
    assert np.max(np.abs(rec - want), axis=0).max() <= 1e-13 * max(1.0, np.abs(want).max())
    if m > 2:
        s = sc.cpu().numpy()[:(2 + nrhs) * (m - 2) * L].reshape(2 + nrhs, m - 2, L)
        df = o["delta_fwd"] if nrhs == 2 else o["delta_fwd"][..., None]
        fwd = np.stack([o["alpha_fwd"][:, 1:m - 1].T, o["gamma_fwd"][:, 1:m - 1].T] +
                       [df[:, 1:m - 1, q].T for q in range(nrhs)])
        assert np.max(np.abs(s - fwd)) <= 1e-13 * max(1.0, np.abs(fwd).max())
