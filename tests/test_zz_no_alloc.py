"""The allocation-free <C> / top-k entry point.

qaoa_expect_topk_static serves callers that cannot allocate device memory (memory owned by
another allocator or a fixed budget, loops that must not synchronise in cudaMalloc, callers
without a qaoa_ctx workspace): its scratch is a fixed array inside the library. This test calls
it through the C ABI and checks, on two calls in a row (the second one reuses the scratch the
first left behind), that it returns what the workspace-based qaoa_expect and qaoa_topk return.
It runs alone in a fresh process as well as after the other tests (it creates its own state).
"""
import ctypes as C

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


def make_state(q, ctx, n, p, seed):
    Q = torch.as_tensor(synth.symmetric_q(n, seed=seed).astype(np.float32)).cuda()
    g, b = synth.random_params(p, seed=seed + 1)
    gd = torch.as_tensor(g.astype(np.float32)).cuda()
    bd = torch.as_tensor(b.astype(np.float32)).cuda()
    E = torch.empty(1 << n, dtype=torch.float32, device="cuda")
    psi = torch.empty(2 << n, dtype=torch.float32, device="cuda")
    q.qaoa_build_energies(ctx, n, Q, E)
    q.qaoa_run_layers(ctx, n, p, gd, bd, E, psi, True)
    return psi, E


def test_static_scratch_matches_workspace_entry_points(q):
    L = q.lib()
    ctx = q.qaoa_create(0)
    try:
        q.qaoa_reserve(ctx, q.qaoa_workspace_bytes(22))
        stream = torch.cuda.current_stream().cuda_stream
        for n, p, k, seed in [(20, 2, 8, 5), (11, 3, 16, 9)]:
            psi, E = make_state(q, ctx, n, p, seed)
            ref_ex = torch.zeros(1, dtype=torch.float64, device="cuda")
            ref_i = torch.zeros(k, dtype=torch.int64, device="cuda")
            ref_p = torch.zeros(k, dtype=torch.float64, device="cuda")
            q.qaoa_expect(ctx, n, psi, E, ref_ex)
            q.qaoa_topk(ctx, n, psi, k, ref_i, ref_p)
            torch.cuda.synchronize()
            absq = float(np.abs(synth.symmetric_q(n, seed=seed)).sum())
            for call in range(2):          # two calls in a row share the fixed scratch
                ex = torch.full((1,), -7.0, dtype=torch.float64, device="cuda")
                ti = torch.full((k,), -1, dtype=torch.int64, device="cuda")
                tp = torch.full((k,), -1.0, dtype=torch.float64, device="cuda")
                st = L.qaoa_expect_topk_static(n, C.c_void_p(psi.data_ptr()), C.c_void_p(E.data_ptr()), k,
                                               C.c_void_p(ex.data_ptr()), C.c_void_p(ti.data_ptr()),
                                               C.c_void_p(tp.data_ptr()), C.c_void_p(stream))
                assert st == q.QAOA_OK, q.qaoa_last_error()
                torch.cuda.synchronize()
                assert abs(ex.item() - ref_ex.item()) <= 1e-5 * absq, (n, call)
                np.testing.assert_array_equal(ti.cpu().numpy(), ref_i.cpu().numpy())
                np.testing.assert_allclose(tp.cpu().numpy(), ref_p.cpu().numpy(), rtol=0, atol=1e-12)
            # optional outputs: top-k alone (expect and E NULL, prob NULL) and <C> alone (k = 0)
            ti2 = torch.full((k,), -1, dtype=torch.int64, device="cuda")
            st = L.qaoa_expect_topk_static(n, C.c_void_p(psi.data_ptr()), None, k, None,
                                           C.c_void_p(ti2.data_ptr()), None, C.c_void_p(stream))
            assert st == q.QAOA_OK, q.qaoa_last_error()
            ex2 = torch.full((1,), -7.0, dtype=torch.float64, device="cuda")
            st = L.qaoa_expect_topk_static(n, C.c_void_p(psi.data_ptr()), C.c_void_p(E.data_ptr()), 0,
                                           C.c_void_p(ex2.data_ptr()), None, None, C.c_void_p(stream))
            assert st == q.QAOA_OK, q.qaoa_last_error()
            torch.cuda.synchronize()
            np.testing.assert_array_equal(ti2.cpu().numpy(), ref_i.cpu().numpy())
            assert abs(ex2.item() - ref_ex.item()) <= 1e-5 * absq
        # sizes beyond the fixed scratch are refused before any launch
        assert L.qaoa_expect_topk_static(31, C.c_void_p(psi.data_ptr()), None, 1, None,
                                         C.c_void_p(ti.data_ptr()), None, None) == q.QAOA_E_INVALID
        assert L.qaoa_expect_topk_static(10, C.c_void_p(psi.data_ptr()), None, 17, None,
                                         C.c_void_p(ti.data_ptr()), None, None) == q.QAOA_E_INVALID
    finally:
        q.qaoa_destroy(ctx)
