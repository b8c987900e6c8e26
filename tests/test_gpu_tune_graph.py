"""Autotuner table (tune, store, save / load as JSON, plans follow it) and CUDA-graph capture of
a plan (replays give the same results as direct launches and pick up new inputs)."""
import json

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def q():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2506_10531_gb300 import build
    build.build()
    import paper_2506_10531_gb300 as qq
    return qq


def batch(q, specs, seed):
    Qs, pars, rows = [], [], []
    qo = po = 0
    for i, (n, p, k) in enumerate(specs):
        Q = synth.symmetric_q(n, seed=seed + i).astype(np.float32)
        g, b = synth.random_params(p, seed=seed + 100 + i)
        Qs.append(Q.reshape(-1))
        pars.append(np.concatenate([g, b]).astype(np.float32))
        rows.append((n, p, k, 0, qo, po, -1, -1))
        qo += n * n
        po += 2 * p
    qd = torch.as_tensor(np.concatenate(Qs)).cuda()
    pd = torch.as_tensor(np.concatenate(pars)).cuda()
    cnt = len(specs)
    ex = torch.zeros(cnt, dtype=torch.float64, device="cuda")
    ti = torch.zeros(cnt * 8, dtype=torch.int64, device="cuda")
    tp = torch.zeros(cnt * 8, dtype=torch.float64, device="cuda")
    io = q.make_io(qd, pd, expect=ex, topk_idx=ti, topk_prob=tp, k_stride=8)
    return q.make_insts(rows), io, pd, (ex, ti, tp)


def test_autotune_table_roundtrip(q, tmp_path):
    ctx = q.qaoa_create(0)
    try:
        ms = q.qaoa_autotune(ctx, 16, 3, 8, 64)
        assert ms > 0
        tier, prm, ms2 = q.qaoa_tuning_get(ctx, 16, 3)
        assert tier in (q.QAOA_TIER_CLUSTER, q.QAOA_TIER_STREAM, q.QAOA_TIER_CSTREAM) and ms2 == pytest.approx(ms)
        if tier == q.QAOA_TIER_CLUSTER:
            assert prm in (13, 14)
        assert q.qaoa_tuning_get(ctx, 16, 4)[0] == 0       # only the tuned shape is stored
        ms_small = q.qaoa_autotune(ctx, 5, 2, 8, 64)        # one configuration: timed, not stored
        assert ms_small > 0 and q.qaoa_tuning_get(ctx, 5, 2)[0] == 0
        path = tmp_path / "tuning.json"
        q.qaoa_tuning_save(ctx, str(path))
        doc = json.loads(path.read_text())
        assert doc["format"] == "libqaoa-tuning-1"
        assert [(e["n"], e["p"], e["tier"]) for e in doc["entries"]] == [(16, 3, tier)]
    finally:
        q.qaoa_destroy(ctx)
    ctx2 = q.qaoa_create(0)
    try:
        q.qaoa_tuning_load(ctx2, str(path))
        assert q.qaoa_tuning_get(ctx2, 16, 3)[:2] == (tier, prm)
        insts, io, _, _ = batch(q, [(16, 3, 8)] * 4, 5)
        plan = q.qaoa_plan_create(ctx2, insts, io)
        try:
            q.qaoa_plan_set_timing(plan, True)
            q.qaoa_plan_launch(plan)
            names = {nm for nm, _ in q.qaoa_plan_kernel_times(plan)}
            assert ("cluster" in names) == (tier == q.QAOA_TIER_CLUSTER)
            assert bool({"stream_pass", "tstream_pass"} & names) == (tier == q.QAOA_TIER_STREAM)
            assert ("cstream" in names) == (tier == q.QAOA_TIER_CSTREAM)
        finally:
            q.qaoa_plan_destroy(plan)
        # an explicit tier setting overrides the table
        q.qaoa_set_tier(ctx2, 16, q.QAOA_TIER_STREAM, 0)
        plan = q.qaoa_plan_create(ctx2, insts, io)
        try:
            q.qaoa_plan_set_timing(plan, True)
            q.qaoa_plan_launch(plan)
            assert {"stream_pass", "tstream_pass"} & {nm for nm, _ in q.qaoa_plan_kernel_times(plan)}
        finally:
            q.qaoa_plan_destroy(plan)
    finally:
        q.qaoa_destroy(ctx2)


def test_plan_graph_capture_replays(q):
    ctx = q.qaoa_create(0)
    specs = [(10, 2, 8), (14, 3, 8), (16, 2, 8), (20, 2, 8), (12, 1, 8), (16, 2, 8)]
    try:
        insts, io, pd, outs = batch(q, specs, 31)
        direct = q.qaoa_plan_create(ctx, insts, io)
        q.qaoa_plan_launch(direct)
        torch.cuda.synchronize()
        ref = [o.clone() for o in outs]
        s = torch.cuda.Stream()
        graph = q.qaoa_plan_create(ctx, insts, io)
        q.qaoa_plan_capture(graph, s)
        for o in outs:
            o.zero_()
        torch.cuda.synchronize()
        for _ in range(2):
            q.qaoa_plan_launch(graph, s)
        s.synchronize()
        for a, b in zip(outs, ref):
            assert torch.equal(a, b)
        # new parameters written into the bound pool are seen by the replay
        pd.mul_(0.5)
        q.qaoa_plan_launch(direct)
        torch.cuda.synchronize()
        ref2 = [o.clone() for o in outs]
        assert not torch.equal(ref2[0], ref[0])
        for o in outs:
            o.zero_()
        torch.cuda.synchronize()
        q.qaoa_plan_launch(graph, s)
        s.synchronize()
        for a, b in zip(outs, ref2):
            assert torch.equal(a, b)
        q.qaoa_plan_destroy(graph)
        q.qaoa_plan_destroy(direct)
    finally:
        q.qaoa_destroy(ctx)


def test_streaming_variants_agree_and_tune(q, tmp_path):
    # the streaming tier's forward-pass variants (TMA passes with two or one CTA per SM, the
    # cp.async passes) give the same results (the two TMA grids bit for bit: same arithmetic per
    # tile, fixed reduction order), and the tuner stores a variant for n = 20 that plans follow
    specs = [(20, 2, 8)] * 3
    out = {}
    for v in (0, 1, 2):
        ctx = q.qaoa_create(0)
        try:
            q.qaoa_set_tier(ctx, 20, q.QAOA_TIER_STREAM, v)
            insts, io, _, (ex, ti, tp) = batch(q, specs, 41)
            plan = q.qaoa_plan_create(ctx, insts, io)
            try:
                q.qaoa_plan_set_timing(plan, True)
                q.qaoa_plan_launch(plan)
                torch.cuda.synchronize()
                names = {nm for nm, _ in q.qaoa_plan_kernel_times(plan)}
                q.qaoa_plan_check(plan)
            finally:
                q.qaoa_plan_destroy(plan)
            out[v] = (ex.cpu().numpy(), ti.cpu().numpy(), tp.cpu().numpy(), names)
        finally:
            q.qaoa_destroy(ctx)
    assert "tstream_pass" in out[0][3] and "tstream_pass" in out[1][3] and "stream_pass" in out[2][3]
    for a, b in zip(out[0][:3], out[1][:3]):
        np.testing.assert_array_equal(a, b)
    absq = max(float(np.abs(synth.symmetric_q(20, seed=41 + i)).sum()) for i in range(3))
    assert np.max(np.abs(out[2][0] - out[0][0])) <= 2e-5 * absq
    assert np.max(np.abs(out[2][2] - out[0][2])) <= 1e-6 * max(out[0][2].max(), 1e-30) + 1e-12
    ctx = q.qaoa_create(0)
    try:
        with pytest.raises(q.QaoaError):
            q.qaoa_set_tier(ctx, 20, q.QAOA_TIER_STREAM, 3)
        ms = q.qaoa_autotune(ctx, 20, 2, 8, 4)
        tier, prm, _ = q.qaoa_tuning_get(ctx, 20, 2)
        assert ms > 0 and tier == q.QAOA_TIER_STREAM and prm in (0, 1, 2)
        path = tmp_path / "tuning20.json"
        q.qaoa_tuning_save(ctx, str(path))
    finally:
        q.qaoa_destroy(ctx)
    ctx = q.qaoa_create(0)
    try:
        q.qaoa_tuning_load(ctx, str(path))
        assert q.qaoa_tuning_get(ctx, 20, 2)[:2] == (tier, prm)
    finally:
        q.qaoa_destroy(ctx)


def test_resident_window_variants_agree_and_tune(q):
    # the resident tier with forward register windows of 5 and 4 qubits (blocks of 2^(n-5) and
    # 2^(n-4) threads) gives the same results within rounding; the tuner stores one for n = 12
    specs = [(12, 3, 8)] * 6 + [(9, 2, 8)] * 3 + [(13, 1, 8)] * 2
    out = {}
    for r in (5, 4):
        ctx = q.qaoa_create(0)
        try:
            for n in (9, 12, 13):
                q.qaoa_set_tier(ctx, n, q.QAOA_TIER_RESIDENT, r)
            insts, io, _, (ex, ti, tp) = batch(q, specs, 61)
            plan = q.qaoa_plan_create(ctx, insts, io)
            try:
                q.qaoa_plan_launch(plan)
                torch.cuda.synchronize()
            finally:
                q.qaoa_plan_destroy(plan)
            out[r] = (ex.cpu().numpy(), ti.cpu().numpy(), tp.cpu().numpy())
        finally:
            q.qaoa_destroy(ctx)
    for i, (n, p, k) in enumerate(specs):
        absq = float(np.abs(synth.symmetric_q(n, seed=61 + i)).sum())
        assert abs(out[5][0][i] - out[4][0][i]) <= 2e-5 * absq, i
        a, b = out[5][2][i * 8:(i + 1) * 8], out[4][2][i * 8:(i + 1) * 8]
        # probabilities of amplitudes within 1e-5 of each other: |dp| <= 2e-5 sqrt(p) + 1e-10
        assert np.max(np.abs(a - b)) <= 2e-5 * np.sqrt(a.max()) + 1e-10, i
    ctx = q.qaoa_create(0)
    try:
        with pytest.raises(q.QaoaError):
            q.qaoa_set_tier(ctx, 12, q.QAOA_TIER_RESIDENT, 3)
        with pytest.raises(q.QaoaError):
            q.qaoa_set_tier(ctx, 14, q.QAOA_TIER_RESIDENT, 4)   # a window would start at bit 10
        ms = q.qaoa_autotune(ctx, 12, 3, 8, 256)
        tier, prm, _ = q.qaoa_tuning_get(ctx, 12, 3)
        assert ms > 0 and tier == q.QAOA_TIER_RESIDENT and prm in (4, 5)
    finally:
        q.qaoa_destroy(ctx)
