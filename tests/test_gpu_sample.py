"""Measurement shots (qaoa_sample) against the FP64 oracle's inverse-CDF sampler on the same
complex64 state and the same uniforms: every shot equal, except where the target lies within
1e-12 of a cumulative-probability boundary (the device sums per part, the oracle in one pass);
there the device's index must still bracket the target."""
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


@pytest.fixture(scope="module")
def ctx(q):
    c = q.qaoa_create(0)
    yield c
    q.qaoa_destroy(c)


def state(q, ctx, n, g, b, seed):
    Q32 = synth.symmetric_q(n, seed=seed).astype(np.float32)
    qd = torch.as_tensor(Q32.reshape(-1)).cuda()
    pd = torch.as_tensor(np.concatenate([g, b]).astype(np.float32)).cuda()
    psi = torch.zeros(2 << n, dtype=torch.float32, device="cuda")
    ex = torch.zeros(1, dtype=torch.float64, device="cuda")
    io = q.make_io(qd, pd, expect=ex, psi=psi)
    q.qaoa_batch_run(ctx, q.make_insts([(n, len(g), 0, 0, 0, 0, 0, -1)]), io)
    torch.cuda.synchronize()
    return psi


def check(orc, psi_dev, u, z_dev):
    ps = psi_dev.cpu().numpy().reshape(-1, 2).astype(np.float64)
    pr = orc.probs(ps[:, 0] + 1j * ps[:, 1])
    zo = orc.sample_probs(pr, u)
    zg = z_dev.cpu().numpy().astype(np.uint64)
    cdf = np.cumsum(pr)
    t = u * cdf[-1]
    tol = 1e-12 * cdf[-1]
    for i in np.nonzero(zg != zo)[0]:
        z = int(zg[i])
        lo = cdf[z - 1] if z > 0 else 0.0
        assert lo - tol <= t[i] < cdf[z] + tol, (i, z, int(zo[i]))
        assert np.min(np.abs(cdf - t[i])) <= tol, i
    return zg, zo


@pytest.mark.parametrize("n", [1, 4, 12, 13, 16, 20])
def test_sample_matches_oracle(q, ctx, orc, n):
    g, b = synth.random_params(2, seed=900 + n)
    psi = state(q, ctx, n, g.astype(np.float32), b.astype(np.float32), 901 + n)
    shots = 4096
    u = synth.uniform01(902 + n, shots)
    ud = torch.as_tensor(u).cuda()
    z = torch.zeros(shots, dtype=torch.int64, device="cuda")
    q.qaoa_sample(ctx, n, psi, shots, ud, z)
    torch.cuda.synchronize()
    zg, zo = check(orc, psi, u, z)
    assert np.mean(zg == zo) > 0.999


def test_sample_uniform_state_and_edges(q, ctx, orc):
    # zero angles keep |+>: shot s is floor(u_s 2^n) up to boundary rounding
    n, shots = 14, 8192
    psi = state(q, ctx, n, np.zeros(1, np.float32), np.zeros(1, np.float32), 950)
    u = synth.uniform01(951, shots)
    ud = torch.as_tensor(u).cuda()
    z = torch.zeros(shots, dtype=torch.int64, device="cuda")
    q.qaoa_sample(ctx, n, psi, shots, ud, z)
    torch.cuda.synchronize()
    zg, _ = check(orc, psi, u, z)
    assert np.mean(zg.astype(np.int64) == np.floor(u * (1 << n)).astype(np.int64)) > 0.999
    # zero shots is a no-op; bad arguments are rejected before any launch
    q.qaoa_sample(ctx, n, psi, 0, None, None)
    with pytest.raises(q.QaoaError):
        q.qaoa_sample(ctx, 31, psi, 1, ud, z)
    with pytest.raises(q.QaoaError):
        q.qaoa_sample(ctx, n, psi, -1, ud, z)
    with pytest.raises(q.QaoaError):
        q.qaoa_sample(ctx, n, psi, 4, None, z)
