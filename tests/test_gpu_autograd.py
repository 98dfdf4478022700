"""Differentiation through the DLT / IDLT (torch.autograd with the library's
transposed kernels as the hand-written backward).

Workload of the differentiation experiment: a batch of 256 coefficient vectors
of N = 4096, loss = ||DLT(c) - y||^2 with y = DLT(c*) + 1e-3 * noise.  The loss
is quadratic, so central differences (h = 1e-6) are exact up to rounding; the
gradient 2 P^T (P c - y) is also checked against the oracle's dense P^T.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ag():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1505_00354_gb300 import build
    build.build()
    from paper_1505_00354_gb300 import autograd
    return autograd


def _batch(B, N, seed, decay=1.0):
    from paper_1505_00354_gb300 import inputs
    return np.stack([inputs.coeffs(N, seed * 1000 + i, decay) for i in range(B)])


def test_dlt_gradient_fd_and_dense(ag):
    import oracle
    B, N = 256, 4096
    cstar = torch.tensor(_batch(B, N, 50), device="cuda")
    noise = torch.tensor(np.random.default_rng(51).standard_normal((B, N)), device="cuda")
    with torch.no_grad():
        y = ag.dlt(cstar) + 1e-3 * noise
    c = torch.tensor(_batch(B, N, 52), device="cuda", requires_grad=True)

    def loss_of(cc):
        return ((ag.dlt(cc) - y) ** 2).sum()

    loss = loss_of(c)
    loss.backward()
    grad = c.grad.detach()
    # central finite differences at 64 seeded coordinates and 8 random directions.
    # The loss is a sum of ~1e6 positive terms; each evaluation carries a
    # rounding error of at most ~log2(terms) * u * loss, so a central difference
    # with step h is exact only to ~2 * 32 * u * loss / (2h) in absolute terms.
    rng = np.random.default_rng(53)
    h = 1e-6
    u = 2.0**-53
    noise = 32 * u * float(loss) / h
    coords = [(int(rng.integers(B)), int(rng.integers(N))) for _ in range(64)]
    with torch.no_grad():
        worst = 0.0
        for b, n in coords:
            e = torch.zeros_like(c)
            e[b, n] = h
            fd = (loss_of(c + e) - loss_of(c - e)).item() / (2 * h)
            worst = max(worst, abs(fd - grad[b, n].item()) / (noise + 1e-7 * abs(fd)))
        for _ in range(8):
            d = torch.tensor(rng.standard_normal((B, N)), device="cuda")
            fd = (loss_of(c + h * d) - loss_of(c - h * d)).item() / (2 * h)
            an = float((grad * d).sum())
            worst = max(worst, abs(fd - an) / (noise + 1e-7 * abs(fd)))
    print(f"FD check: loss {float(loss):.3e}, rounding bound {noise:.2e}, worst |fd - grad| / bound {worst:.2f}")
    assert worst <= 1.0
    # dense P^T g from the oracle for a few batch rows
    nd = oracle.legpts(N)
    with torch.no_grad():
        r = (ag.dlt(c) - y).cpu().numpy()
    for b in (0, 17, 255):
        ref = 2.0 * oracle.dlt_t(r[b], nd)
        got = grad[b].cpu().numpy()
        err = np.max(np.abs(got - ref)) / np.abs(2.0 * r[b]).sum()
        print(f"row {b}: |grad - 2 P^T r| / ||2 r||_1 = {err:.2e}")
        assert err <= 1e-12


def test_idlt_gradient_matches_transpose(ag):
    """<IDLT(f), g> = <f, IDLT^T(g)>: backward of the IDLT through autograd."""
    N = 1024
    f = torch.tensor(np.random.default_rng(60).standard_normal((4, N)), device="cuda", requires_grad=True)
    g = torch.tensor(np.random.default_rng(61).standard_normal((4, N)), device="cuda")
    (ag.idlt(f) * g).sum().backward()
    from paper_1505_00354_gb300 import get_plan, FP64
    p = get_plan(N, FP64)
    ref = p.idlt_t(g)
    assert torch.allclose(f.grad, ref, rtol=0, atol=1e-12 * float(ref.abs().max()))


def test_gradcheck_small(ag):
    c = torch.tensor(np.random.default_rng(70).standard_normal((2, 32)), device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(ag.dlt, (c,), eps=1e-6, atol=1e-8, rtol=1e-7)
    f = torch.tensor(np.random.default_rng(71).standard_normal((2, 32)), device="cuda", requires_grad=True)
    assert torch.autograd.gradcheck(ag.idlt, (f,), eps=1e-6, atol=1e-8, rtol=1e-7)


def test_fp32_gradients_vs_oracle(ag):
    """The FP32 form through autograd: the DLT's gradient 2 P^T r and the IDLT's
    vector-Jacobian product D_w P D_s g against the oracle, at the FP32 form's
    bar (5e-6 in the ||c||_1 normalisation)."""
    import oracle
    N, B = 4096, 4
    nd = oracle.legpts(N)
    c = torch.tensor(_batch(B, N, 80), dtype=torch.float32, device="cuda", requires_grad=True)
    y = torch.tensor(_batch(B, N, 81, decay=0.0), dtype=torch.float32, device="cuda")
    loss = ((ag.dlt(c) - y) ** 2).sum()
    loss.backward()
    with torch.no_grad():
        r = (ag.dlt(c) - y).double().cpu().numpy()
    grad = c.grad.double().cpu().numpy()
    for b in range(B):
        rb = r[b].astype(np.float32).astype(np.float64)
        ref = 2.0 * oracle.dlt_t(rb, nd)
        err = np.max(np.abs(grad[b] - ref)) / np.abs(2.0 * rb).sum()
        assert err <= 5e-6, (b, err)
    f = torch.tensor(np.random.default_rng(82).standard_normal((B, N)), dtype=torch.float32, device="cuda",
                     requires_grad=True)
    g = torch.tensor(np.random.default_rng(83).standard_normal((B, N)), dtype=torch.float32, device="cuda")
    (ag.idlt(f) * g).sum().backward()
    gd = g.double().cpu().numpy()
    for b in range(B):
        sg = (np.arange(N) + 0.5) * gd[b]
        ref = nd.w * oracle.dlt_rows(sg, nd)
        err = np.max(np.abs(f.grad[b].double().cpu().numpy() - ref)) / np.abs(sg).sum()
        assert err <= 5e-6, (b, err)
