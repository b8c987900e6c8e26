"""Serving: continuous batching of optimise-and-sample jobs through the C ABI.

* A job's result (final parameters, <C>, top-k) is bit-for-bit the same alone and in a mix of
  other jobs that arrive before, with and after it (batch-invariant kernels, per-job Adam).
* It equals the same optimisation run as a one-instance training batch (plan launch + Adam
  kernel per step) followed by a forward pass with top-k.
* Admission respects the scratch budget (jobs wait in the queue), every job completes, and each
  final <C> and top-k matches the FP64 oracle at the returned parameters.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

K = 8


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_10531_gb300 import build
    build.build()
    import paper_2506_10531_gb300 as qq
    return qq


@pytest.fixture(scope="module")
def ctx(q):
    c = q.qaoa_create(0)
    yield c
    q.qaoa_destroy(c)


def job(n, p, seed, steps=6):
    Q = synth.symmetric_q(n, seed=seed).astype(np.float32)
    g, b = synth.random_params(p, seed=seed + 1)
    return dict(n=n, p=p, Q=Q, params=np.concatenate([g, b]).astype(np.float32), steps=steps, lr=0.05)


def run_server(q, ctx, schedule, scratch=8 << 30, max_jobs=64):
    """schedule: list of (tick at which to submit, job dict). Returns {index: result}."""
    srv = q.qaoa_server_create(ctx, scratch, max_jobs, K)
    try:
        ids, out = {}, {}
        t = 0
        while len(out) < len(schedule):
            for i, (at, jb) in enumerate(schedule):
                if at == t:
                    ids[q.qaoa_server_submit(srv, jb["n"], jb["p"], jb["Q"], jb["params"], jb["steps"], jb["lr"])] = i
            q.qaoa_server_tick(srv)
            for r in q.qaoa_server_poll(srv, wait=True):
                out[ids[r.job_id]] = r
            t += 1
            assert t < 1000
        return out
    finally:
        q.qaoa_server_destroy(srv)


def as_tuple(r):
    p = r.p
    return (r.expect, tuple(r.topk_idx[:K]), tuple(r.topk_prob[:K]), tuple(r.params[:2 * p]))


def test_alone_equals_mixed(q, ctx):
    J = job(16, 2, 101, steps=7)
    alone = run_server(q, ctx, [(0, J)])[0]
    others = [job(10, 3, 201, 4), job(19, 1, 202, 9), job(14, 2, 203, 5), job(12, 4, 204, 3),
              job(21, 2, 205, 6), job(16, 2, 206, 8)]
    sched = [(0, others[0]), (0, others[1]), (2, others[2]), (3, J), (3, others[3]), (5, others[4]),
             (9, others[5])]
    mixed = run_server(q, ctx, sched)
    assert as_tuple(mixed[3]) == as_tuple(alone)


def test_server_equals_training_batch(q, ctx):
    from paper_2506_10531_gb300.train import QAOABatch, adam_train
    J = job(17, 3, 301, steps=5)
    r = run_server(q, ctx, [(0, J)])[0]
    g0, b0 = J["params"][:3], J["params"][3:]
    B = QAOABatch(ctx, [J["Q"]], [(g0, b0)])
    try:
        adam_train(B, J["steps"], J["lr"])
        torch.cuda.synchronize()
        par = B.params.cpu().numpy()
    finally:
        B.close()
    np.testing.assert_array_equal(np.array(r.params[:6], dtype=np.float32), par)
    # final forward with top-k at those parameters
    qd = torch.as_tensor(J["Q"].reshape(-1)).cuda()
    pd = torch.as_tensor(par).cuda()
    ex = torch.zeros(1, dtype=torch.float64, device="cuda")
    ti = torch.zeros(K, dtype=torch.int64, device="cuda")
    tp = torch.zeros(K, dtype=torch.float64, device="cuda")
    io = q.make_io(qd, pd, expect=ex, topk_idx=ti, topk_prob=tp, k_stride=K)
    q.qaoa_batch_run(ctx, q.make_insts([(17, 3, K, 0, 0, 0, -1, -1)]), io)
    torch.cuda.synchronize()
    assert r.expect == ex.item()
    assert list(r.topk_idx[:K]) == [int(v) for v in ti.cpu().numpy()]
    assert list(r.topk_prob[:K]) == list(tp.cpu().numpy())


def test_admission_budget_and_oracle(q, ctx, orc):
    jobs = [job(20, 2, 401 + i, steps=3) for i in range(5)] + [job(11, 2, 420, steps=2)]
    srv = q.qaoa_server_create(ctx, 0, 16, K)   # zero scratch: streaming jobs never fit
    try:
        with pytest.raises(q.QaoaError):
            q.qaoa_server_submit(srv, 20, 2, jobs[0]["Q"], jobs[0]["params"], 3, 0.05)
    finally:
        q.qaoa_server_destroy(srv)
    per_job = None
    srv = q.qaoa_server_create(ctx, 1, 1, K)
    try:
        per_job = q.qaoa_server_job_bytes(srv, 20, 2)
    finally:
        q.qaoa_server_destroy(srv)
    srv = q.qaoa_server_create(ctx, 2 * per_job + 4096, 16, K)   # room for two n = 20 jobs
    try:
        ids = {q.qaoa_server_submit(srv, j["n"], j["p"], j["Q"], j["params"], j["steps"], j["lr"]): i
               for i, j in enumerate(jobs)}
        active, queued = q.qaoa_server_tick(srv)
        # two n = 20 jobs fit; the small resident job waits behind the queue head (FIFO)
        assert active == 2 and queued == 4
        out = {}
        for _ in range(200):
            q.qaoa_server_tick(srv)
            qs, act, used, _, _, _ = q.qaoa_server_stats(srv)
            assert used <= 2 * per_job + 4096
            for r in q.qaoa_server_poll(srv, wait=True):
                out[ids[r.job_id]] = r
            if len(out) == len(jobs):
                break
        assert len(out) == len(jobs)
    finally:
        q.qaoa_server_destroy(srv)
    for i, j in enumerate(jobs):
        r = out[i]
        n, p = j["n"], j["p"]
        par = np.array(r.params[:2 * p], dtype=np.float32).astype(np.float64)
        Qd = j["Q"].astype(np.float64)
        E = orc.energies(Qd)
        psi = orc.state(n, par[:p], par[p:], E)
        absq = np.abs(Qd).sum()
        assert abs(r.expect - orc.expect(psi, E)) <= 1e-5 * absq
        pr = orc.probs(psi)
        _, rp = orc.topk_probs(pr, K)
        got = np.array(r.topk_prob[:K])
        assert np.all(np.abs(got - rp) <= 4e-5 * np.sqrt(rp[0]))
        for z, pz in zip(r.topk_idx[:K], got):
            assert abs(pr[int(z)] - pz) <= 4e-5 * np.sqrt(rp[0])


def same_result(a, b):
    assert a.expect == b.expect
    np.testing.assert_array_equal(np.array(a.topk_idx[:K]), np.array(b.topk_idx[:K]))
    np.testing.assert_array_equal(np.array(a.params[:2 * a.p]), np.array(b.params[:2 * b.p]))


def test_cancel_queued_and_running_jobs(q, ctx):
    # host-side failure handling: a queued job and a running job are withdrawn; the others
    # finish with the results they have alone, and the withdrawn ones never report
    jobs = [job(10, 2, 501, steps=5), job(14, 3, 502, steps=8), job(12, 2, 503, steps=8), job(16, 1, 504, steps=4)]
    srv = q.qaoa_server_create(ctx, 8 << 30, 2, K)   # two slots: jobs 2 and 3 wait in the queue
    try:
        ids = [q.qaoa_server_submit(srv, jb["n"], jb["p"], jb["Q"], jb["params"], jb["steps"], jb["lr"]) for jb in jobs]
        q.qaoa_server_tick(srv)                       # admits jobs 0 and 1
        q.qaoa_server_cancel(srv, ids[2])             # queued
        q.qaoa_server_cancel(srv, ids[1])             # running: its slot goes to job 3
        with pytest.raises(q.QaoaError):
            q.qaoa_server_cancel(srv, ids[2])         # already gone
        with pytest.raises(q.QaoaError):
            q.qaoa_server_cancel(srv, 10 ** 9)        # unknown
        out = {}
        for _ in range(60):
            a, qd = q.qaoa_server_tick(srv)
            for r in q.qaoa_server_poll(srv, wait=True):
                out[r.job_id] = r
            if len(out) == 2 and a == 0 and qd == 0:
                break
        queued, active, used, _, _, _ = q.qaoa_server_stats(srv)
        assert queued == 0 and active == 0 and used == 0
        for r in q.qaoa_server_poll(srv, wait=True):
            out[r.job_id] = r
    finally:
        q.qaoa_server_destroy(srv)
    assert sorted(out) == sorted([ids[0], ids[3]])
    alone0 = run_server(q, ctx, [(0, jobs[0])])[0]
    alone3 = run_server(q, ctx, [(0, jobs[3])])[0]
    same_result(out[ids[0]], alone0)
    same_result(out[ids[3]], alone3)


def test_admission_failure_injected(q, ctx):
    # the next two admission attempts fail as if the job's scratch could not be allocated: the
    # job keeps its place, admission resumes after two ticks, and every result is unchanged
    jobs = [job(11, 2, 511, steps=3), job(13, 2, 512, steps=3), job(15, 1, 513, steps=2)]
    srv = q.qaoa_server_create(ctx, 8 << 30, 8, K)
    try:
        ids = [q.qaoa_server_submit(srv, jb["n"], jb["p"], jb["Q"], jb["params"], jb["steps"], jb["lr"]) for jb in jobs]
        assert q.qaoa_server_fail_admissions(srv, 2) == 0
        assert q.qaoa_server_tick(srv) == (0, 3)
        assert q.qaoa_server_tick(srv) == (0, 3)
        assert q.qaoa_server_fail_admissions(srv, 0) == 2
        assert q.qaoa_server_tick(srv) == (3, 0)
        out = {}
        for _ in range(40):
            q.qaoa_server_tick(srv)
            for r in q.qaoa_server_poll(srv, wait=True):
                out[r.job_id] = r
            if len(out) == 3:
                break
    finally:
        q.qaoa_server_destroy(srv)
    ref = run_server(q, ctx, [(0, jb) for jb in jobs])
    for i in range(3):
        same_result(out[ids[i]], ref[i])
