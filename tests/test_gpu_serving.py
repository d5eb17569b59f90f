"""Serving: continuous batching of solves on resident hierarchies (C ABI nmg_server_*).

Each request's result must be the same alone (nmg_solve) and in a mix of
concurrently running requests of different meshes; the kernels are
deterministic, so the expected agreement is bitwise.
"""

import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from gen import Problem, build_system

pytestmark = pytest.mark.gpu

MESHES = [
    Problem(dim=2, n=(32, 32), levels=3, solid=(0, +1, 0.6), conv_seed=10),
    Problem(dim=2, n=(64, 64), levels=4, solid=(0, +1, 0.6), conv_seed=12),
    Problem(dim=2, n=(24, 40), levels=3, solid=(0, +1, 0.6), conv_seed=14),
    Problem(dim=3, n=(8, 8, 8), levels=2, solid=(2, -1, 0.25), conv_seed=16),
    Problem(dim=3, n=(16, 16, 16), levels=3, solid=(2, -1, 0.25), conv_seed=18),
]


@pytest.fixture(scope="module")
def pool():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1904_02401_gb300.session import Session
    out = []
    for p in MESHES:
        s = build_system(p)
        S = Session(p.dim, p.n, [(l.row_ptr, l.col_idx, l.vals) for l in s.levels], s.dirichlet,
                    precisions=(1 << 0) | (1 << 1))
        out.append((s, S))
    yield out
    for _, S in out:
        S.close()


def _rhs(s, seed):
    rng = np.random.default_rng(seed)
    b = rng.uniform(-1.0, 1.0, s.unknowns)
    b[s.dirichlet.astype(bool)] = 0.0
    return torch.from_numpy(b).cuda()


def test_results_identical_alone_and_in_the_mix(pool):
    from paper_1904_02401_gb300 import nmg
    from paper_1904_02401_gb300.session import solve_opts
    reqs = []
    for i in range(20):
        k = i % len(pool)
        prec = (1, 0)[i % 2]
        reqs.append((k, prec, 100 + i))
    # alone
    alone = []
    for k, prec, seed in reqs:
        s, S = pool[k]
        b = _rhs(s, seed)
        x = torch.empty_like(b)
        info = S.solve(b, x, precision=prec, engine=nmg.NMG_ENGINE_KERNELS)
        assert info.status == 0
        alone.append((x.clone(), info.iterations))
    # in the mix
    server = C.c_void_p()
    nmg.check(nmg.nmg_server_create(0, 4, server))
    try:
        bufs, tickets = [], []
        for k, prec, seed in reqs:
            s, S = pool[k]
            b = _rhs(s, seed)
            x = torch.zeros_like(b)
            bufs.append((b, x))
        torch.cuda.synchronize()
        for (k, prec, seed), (b, x) in zip(reqs, bufs):
            t = C.c_uint64()
            nmg.check(nmg.nmg_submit(server, pool[k][1].handle, b, x,
                                     solve_opts(precision=prec, engine=nmg.NMG_ENGINE_KERNELS), t))
            tickets.append(t.value)
        for i, t in enumerate(tickets):
            info = nmg.nmg_solve_info()
            st = nmg.nmg_poll(server, t, 60000, info)
            assert st == 0, (st, nmg.nmg_last_error())
            x = bufs[i][1]
            assert torch.equal(x, alone[i][0]), i
            assert info.iterations == alone[i][1]
            assert info.ms_total > 0
        # a released ticket is unknown afterwards
        assert nmg.nmg_poll(server, tickets[0], 0, None) == nmg.NMG_ERR_INVALID
    finally:
        nmg.nmg_server_destroy(server)


def test_memory_budget_admission(pool):
    from paper_1904_02401_gb300 import nmg
    from paper_1904_02401_gb300.session import solve_opts
    sizes = [S.bytes() for _, S in pool]
    # budget fits the largest hierarchy alone: requests still all complete (one at a time when needed)
    server = C.c_void_p()
    nmg.check(nmg.nmg_server_create(max(sizes), 8, server))
    try:
        bufs, tickets = [], []
        for i, (s, S) in enumerate(pool):
            b = _rhs(s, 7 + i)
            x = torch.zeros_like(b)
            bufs.append((b, x, s, S))
        torch.cuda.synchronize()
        for b, x, s, S in bufs:
            t = C.c_uint64()
            nmg.check(nmg.nmg_submit(server, S.handle, b, x, solve_opts(precision=1), t))
            tickets.append(t.value)
        for t, (b, x, s, S) in zip(tickets, bufs):
            info = nmg.nmg_solve_info()
            assert nmg.nmg_poll(server, t, 60000, info) == 0
            assert info.rel_residual <= 1e-8
    finally:
        nmg.nmg_server_destroy(server)
    # a hierarchy larger than the budget is refused at submission
    server = C.c_void_p()
    nmg.check(nmg.nmg_server_create(min(sizes) // 2, 2, server))
    try:
        s, S = pool[0]
        b = _rhs(s, 1)
        x = torch.zeros_like(b)
        t = C.c_uint64()
        assert nmg.nmg_submit(server, S.handle, b, x, solve_opts(), t) == nmg.NMG_ERR_OOM
    finally:
        nmg.nmg_server_destroy(server)


def test_budget_holds_while_fresh_hierarchies_allocate(pool):
    """Two fresh hierarchies (no solve yet, so no Krylov bases) whose operators
    and workspaces fit the budget together, but not once both have allocated
    their FGMRES(30) bases: the server runs them one after the other, and the
    resident bytes it reports never exceed the budget.  Both results equal
    nmg_solve's bit for bit."""
    from paper_1904_02401_gb300 import nmg
    from paper_1904_02401_gb300.session import Session, solve_opts
    p = Problem(dim=2, n=(64, 64), levels=4, solid=(0, +1, 0.6), conv_seed=20)
    s = build_system(p)
    lv = [(l.row_ptr, l.col_idx, l.vals) for l in s.levels]
    fresh = [Session(2, p.n, lv, s.dirichlet, precisions=1 << 1) for _ in range(2)]
    alone = Session(2, p.n, lv, s.dirichlet, precisions=1 << 1)
    try:
        krylov = (2 * 30 + 1) * s.unknowns * 8
        size0 = fresh[0].bytes()
        budget = 2 * size0 + krylov   # room for one set of bases only
        o = solve_opts(precision=1, engine=nmg.NMG_ENGINE_KERNELS, use_graph=1)
        server = C.c_void_p()
        nmg.check(nmg.nmg_server_create(budget, 8, server))
        try:
            bufs, tickets = [], []
            for i, S in enumerate(fresh):
                b = _rhs(s, 40 + i)
                x = torch.zeros_like(b)
                bufs.append((b, x))
            torch.cuda.synchronize()
            for S, (b, x) in zip(fresh, bufs):
                t = C.c_uint64()
                nmg.check(nmg.nmg_submit(server, S.handle, b, x, o, t))
                tickets.append(t.value)
            for t in tickets:
                info = nmg.nmg_solve_info()
                assert nmg.nmg_poll(server, t, 60000, info) == 0
            resident, peak = C.c_size_t(), C.c_size_t()
            nmg.check(nmg.nmg_server_memory(server, resident, peak))
            assert size0 + krylov <= peak.value <= budget, (peak.value, budget)
        finally:
            nmg.nmg_server_destroy(server)
        for S, (b, x) in zip(fresh, bufs):
            assert S.bytes() == size0 + krylov                  # each now holds its bases
            ref = torch.zeros_like(b)
            alone.solve(b, ref, precision=1, engine=nmg.NMG_ENGINE_KERNELS, use_graph=1)
            assert torch.equal(ref, x)
    finally:
        for S in fresh + [alone]:
            S.close()


def test_same_hierarchy_requests_overlap(pool):
    """With extra workspaces allowed, requests on one hierarchy run at the same
    time on workspace clones (own vectors and stream, shared matrices and
    inverses); every result is
    bitwise the one nmg_solve gives alone, and the mixed-precision and FP64
    requests on the same clone keep their own iteration counts."""
    from paper_1904_02401_gb300 import nmg
    from paper_1904_02401_gb300.session import solve_opts
    s, S = pool[1]
    reqs = [((1, 0)[i % 3 == 0], 300 + i) for i in range(12)]
    alone = []
    for prec, seed in reqs:
        b = _rhs(s, seed)
        x = torch.empty_like(b)
        info = S.solve(b, x, precision=prec, engine=nmg.NMG_ENGINE_KERNELS)
        assert info.status == 0
        alone.append((x.clone(), info.iterations))
    server = C.c_void_p()
    nmg.check(nmg.nmg_server_create(0, 6, server))
    nmg.check(nmg.nmg_server_set_workspaces(server, 5))
    assert nmg.nmg_server_set_workspaces(server, -1) == nmg.NMG_ERR_INVALID
    try:
        for rnd in range(2):   # the second round reuses the clones the first one made
            bufs, tickets = [], []
            for prec, seed in reqs:
                b = _rhs(s, seed)
                bufs.append((b, torch.zeros_like(b)))
            torch.cuda.synchronize()
            for (prec, seed), (b, x) in zip(reqs, bufs):
                t = C.c_uint64()
                nmg.check(nmg.nmg_submit(server, S.handle, b, x,
                                         solve_opts(precision=prec, engine=nmg.NMG_ENGINE_KERNELS), t))
                tickets.append(t.value)
            for i, t in enumerate(tickets):
                info = nmg.nmg_solve_info()
                assert nmg.nmg_poll(server, t, 60000, info) == 0, nmg.nmg_last_error()
                assert torch.equal(bufs[i][1], alone[i][0]), (rnd, i)
                assert info.iterations == alone[i][1]
    finally:
        nmg.nmg_server_destroy(server)


def test_batched_columns(pool):
    """With batching on, FP32 requests on one hierarchy run as the columns of a
    multi-vector solve (joining while others iterate, leaving when done), FP64
    requests and requests with other V-cycle options wait for their turn, and
    every result and iteration count is bitwise the one nmg_solve gives alone."""
    import time

    from paper_1904_02401_gb300 import nmg
    from paper_1904_02401_gb300.session import solve_opts
    picks = [0, 1, 4]
    reqs = []
    for i in range(22):
        m = picks[i % 3]
        prec = 0 if i % 7 == 3 else 1
        omega = 0.7 if i % 5 == 4 else 0.8
        rtol = 1e-6 if i % 4 == 1 else 1e-8
        reqs.append((m, prec, omega, rtol, 500 + i))
    alone = []
    for m, prec, omega, rtol, seed in reqs:
        s, S = pool[m]
        b = _rhs(s, seed)
        x = torch.empty_like(b)
        info = S.solve(b, x, precision=prec, omega=omega, rtol=rtol, engine=nmg.NMG_ENGINE_KERNELS)
        assert info.status == 0
        alone.append((x.clone(), info.iterations))
    server = C.c_void_p()
    nmg.check(nmg.nmg_server_create(0, 16, server))
    assert nmg.nmg_server_set_batching(server, 9) == nmg.NMG_ERR_INVALID
    nmg.check(nmg.nmg_server_set_batching(server, 8))
    try:
        for rnd in range(2):
            bufs, tickets = [], []
            for m, prec, omega, rtol, seed in reqs:
                b = _rhs(pool[m][0], seed)
                bufs.append((b, torch.zeros_like(b)))
            torch.cuda.synchronize()
            for i, ((m, prec, omega, rtol, seed), (b, x)) in enumerate(zip(reqs, bufs)):
                t = C.c_uint64()
                nmg.check(nmg.nmg_submit(server, pool[m][1].handle, b, x,
                                         solve_opts(precision=prec, omega=omega, rtol=rtol), t))
                tickets.append(t.value)
                if rnd == 1 and i % 6 == 5:
                    time.sleep(0.002)   # later requests join groups that are already iterating
            for i, t in enumerate(tickets):
                info = nmg.nmg_solve_info()
                assert nmg.nmg_poll(server, t, 60000, info) == 0, nmg.nmg_last_error()
                assert info.iterations == alone[i][1], (rnd, i)
                assert torch.equal(bufs[i][1], alone[i][0]), (rnd, i)
    finally:
        nmg.nmg_server_destroy(server)
