"""The differentiable Legendre stage (paper_0910_5435_gb300.autograd): its
hand-written backward (the transposed butterfly) against central finite
differences and against the float64 oracle gradient.

Loss: L(beta) = sum |S beta - g|^2 over G (complex entries independent), so
the exact gradient in PyTorch's convention (dL/dRe + i dL/dIm) is
2 S^T (S beta - g); the oracle evaluates it with its own direct transform
and adjoint, order by order (the map is block diagonal in m).
"""

import numpy as np
import pytest

import oracle
from paper_0910_5435_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 2: 1e-9, 3: 1e-9, 1: 2e-5}


@pytest.fixture(scope="module")
def mods():
    import __graft_entry__
    __graft_entry__.build()
    from paper_0910_5435_gb300 import autograd, sht
    assert torch.cuda.is_available()
    return sht, autograd


def test_gradcheck_small(mods):
    """torch.autograd.gradcheck (finite differences of the forward against
    the backward) on one field and on a batch of three, float64."""
    sht, ag = mods
    P = sht.Plan(6, 1e-12, leaf_cols=4)
    T = inputs.triangle_size(6)
    b1 = torch.from_numpy(inputs.random_beta(6, seed=1)).cuda().requires_grad_()
    assert torch.autograd.gradcheck(lambda b: ag.legendre_synthesis(b, P, 0), (b1,), eps=1e-6, atol=1e-8)
    b3 = torch.from_numpy(np.stack([inputs.random_beta(6, seed=s) for s in (2, 3, 4)])).cuda().requires_grad_()
    assert b3.shape == (3, T)
    assert torch.autograd.gradcheck(lambda b: ag.legendre_synthesis(b, P, 0), (b3,), eps=1e-6, atol=1e-8)


@pytest.fixture(scope="module")
def config512(mods):
    """l = 512, a batch of 16 fields, target g = synthesis of an independent
    beta_g (band-limited), beta and beta_g ~ N(0,1)/(k+1)."""
    sht, ag = mods
    l, nb = 512, 16
    P = sht.Plan(l, 1e-12, leaf_cols=32)
    beta = np.stack([inputs.random_beta(l, seed=5000 + f, decay=True) for f in range(nb)])
    beta_g = np.stack([inputs.random_beta(l, seed=6000 + f, decay=True) for f in range(nb)])
    return P, beta, beta_g


@pytest.mark.parametrize("prec", [0, 2, 3])
def test_gradient_matches_oracle_l512_batch16(mods, config512, prec):
    sht, ag = mods
    P, beta_h, beta_g_h = config512
    l = P.l
    P.prepare(prec)
    g = ag.legendre_synthesis(torch.from_numpy(beta_g_h).cuda(), P, prec).detach()
    beta = torch.from_numpy(beta_h).cuda().requires_grad_()
    loss = (ag.legendre_synthesis(beta, P, prec) - g).abs().pow(2).sum()
    loss.backward()
    torch.cuda.synchronize()
    grad = beta.grad.cpu().numpy()
    off = oracle.triangle_offsets(l)
    ms = [0, 1, 300, 511, 700, 1023]
    sel = np.concatenate([np.arange(off[m], off[m + 1]) for m in ms])
    gh = g.cpu().numpy()
    for f in (0, 15):
        r = oracle.legendre_synthesis(beta_h[f], l, orders=ms) - gh[f]
        r[[m for m in range(2 * l) if m not in ms]] = 0
        ref = 2.0 * oracle.legendre_adjoint(r, l, orders=ms)
        err = np.linalg.norm(grad[f][sel] - ref[sel]) / np.linalg.norm(ref[sel])
        assert err < TOL[prec], (f, err)


def test_gradient_matches_central_differences_l512_batch16(mods, config512):
    """Central differences, h = 1e-6, on 64 random coordinates (real or
    imaginary part of a coefficient of any field), float64 path."""
    sht, ag = mods
    P, beta_h, beta_g_h = config512
    l = P.l
    g = ag.legendre_synthesis(torch.from_numpy(beta_g_h).cuda(), P, 0).detach()
    beta = torch.from_numpy(beta_h).cuda()

    with torch.no_grad():
        base = (ag.legendre_synthesis(beta, P, 0) - g).abs().pow(2)

    def L(b):
        # L(b) - L(beta), summed term by term: only the rows of the perturbed
        # order differ, so the difference carries no cancellation of the
        # whole sum
        with torch.no_grad():
            return float(((ag.legendre_synthesis(b, P, 0) - g).abs().pow(2) - base).sum())

    bg = beta.clone().requires_grad_()
    (ag.legendre_synthesis(bg, P, 0) - g).abs().pow(2).sum().backward()
    grad = bg.grad
    rng = np.random.default_rng(7)
    T = beta.shape[1]
    h = 1e-6
    scale = float(grad.abs().max())
    worst = 0.0
    for _ in range(64):
        f, j, part = int(rng.integers(16)), int(rng.integers(T)), int(rng.integers(2))
        e = torch.zeros_like(beta)
        e[f, j] = h if part == 0 else 1j * h
        fd = (L(beta + e) - L(beta - e)) / (2 * h)
        an = float(grad[f, j].real if part == 0 else grad[f, j].imag)
        worst = max(worst, abs(fd - an) / (abs(an) + 1e-6 * scale))
    assert worst < 1e-6, worst


def test_backward_saves_nothing_but_the_plan(mods):
    """The backward needs no saved tensors (the map is linear)."""
    sht, ag = mods
    P = sht.Plan(8, 1e-12, leaf_cols=4)
    beta = torch.from_numpy(inputs.random_beta(8, seed=9)).cuda().requires_grad_()
    G = ag.legendre_synthesis(beta, P, 0)
    assert len(G.grad_fn.saved_tensors) == 0


def test_checked_launches_raise_on_timeout(mods):
    """check=True reads the device status after the forward and backward
    launches: a sound plan passes both; a plan whose first op waits for a
    completion that never comes raises SHT_ERR_TIMEOUT from the forward."""
    sht, ag = mods
    l = 16
    good = sht.Plan(l, 1e-12, leaf_cols=4)
    bad = sht.Plan(l, 1e-12, leaf_cols=4, debug_unmet_dependency=1)
    b = torch.from_numpy(inputs.random_beta(l, seed=77)).cuda().requires_grad_(True)
    ag.legendre_synthesis(b, good, 0, check=True).abs().pow(2).sum().backward()
    assert b.grad is not None and torch.isfinite(torch.view_as_real(b.grad)).all()
    with pytest.raises(sht.ShtError) as e:
        ag.legendre_synthesis(b.detach(), bad, 0, check=True)
    assert e.value.code == 5
    good.close()
    bad.close()
