"""Batched Legendre stage (sht_batch_*): many fields, each with its own plan
and bandlimit, in one launch, through the C ABI.

The batch runs the same op streams with the same per-op arithmetic as the
single-field entry points, so its outputs equal theirs exactly; a few fields
are also checked against the float64 oracle (tolerances as in the parity
tests: float64 1e-10, split float32 1e-9, float32 2e-5, relative l2).
"""

import numpy as np
import pytest

import oracle
from paper_0910_5435_gb300 import inputs

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

TOL = {0: 1e-10, 2: 1e-9, 3: 1e-9, 1: 2e-5}
CDT = {0: torch.complex128, 2: torch.complex128, 3: torch.complex128, 1: torch.complex64}
LS = (4, 16, 32, 64, 128)


@pytest.fixture(scope="module")
def sht():
    import __graft_entry__
    __graft_entry__.build()
    from paper_0910_5435_gb300 import sht as _sht
    assert torch.cuda.is_available()
    return _sht


@pytest.fixture(scope="module")
def plans(sht):
    return {l: sht.Plan(l, 1e-12, leaf_cols=16) for l in LS}


def rel(a, b):
    a = torch.as_tensor(a).to(torch.complex128).cpu()
    b = torch.as_tensor(b).to(torch.complex128).cpu()
    return float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(b))


def fields(ls, prec, seed):
    betas = [torch.from_numpy(inputs.random_beta(l, seed=seed + f, decay=True)).to(CDT[prec]).cuda()
             for f, l in enumerate(ls)]
    Gs = [torch.full((2 * l, 2 * l), float("nan"), dtype=CDT[prec], device="cuda") for l in ls]
    return betas, Gs


def field_ls(n, seed):
    return [int(x) for x in np.random.default_rng(seed).choice(LS, size=n)]


@pytest.mark.parametrize("prec", [0, 2, 3, 1])
def test_batch_equals_per_field_calls_and_oracle(sht, plans, prec):
    ls = field_ls(11, 4)
    for l in set(ls):
        plans[l].prepare(prec)
    B = sht.Batch([plans[l] for l in ls], prec)
    betas, Gs = fields(ls, prec, 1000)
    bp, gp = sht.pointer_array(betas), sht.pointer_array(Gs)
    sht.sht_batch_synthesize(B, bp, gp)
    assert sht.sht_batch_last_device_status(B) == 0
    for l, beta, G in zip(ls, betas, Gs):
        ref = torch.full_like(G, float("nan"))
        sht.sht_legendre_synthesize(plans[l], prec, beta, ref)
        torch.cuda.synchronize()
        assert torch.equal(G, ref), l
    for f in (0, len(ls) - 1):
        l = ls[f]
        assert rel(Gs[f], oracle.legendre_synthesis(betas[f].cpu().numpy().astype(np.complex128), l)) < TOL[prec]
    # analysis of the fields just synthesized
    backs = [torch.full_like(b, float("nan")) for b in betas]
    sht.sht_batch_analyze(B, gp, sht.pointer_array(backs))
    assert sht.sht_batch_last_device_status(B) == 0
    for l, G, back in zip(ls, Gs, backs):
        ref = torch.full_like(back, float("nan"))
        sht.sht_legendre_analyze(plans[l], prec, G, ref)
        torch.cuda.synchronize()
        assert torch.equal(back, ref), l
    for f, l in enumerate(ls):
        assert rel(backs[f], betas[f]) < 2 * TOL[prec]
    B.close()


def test_batch_in_cuda_graph(sht, plans):
    """The batched launch captured in a CUDA graph and replayed on new inputs
    written into the same buffers."""
    ls = field_ls(7, 5)
    B = sht.Batch([plans[l] for l in ls], 0)
    betas, Gs = fields(ls, 0, 2000)
    bp, gp = sht.pointer_array(betas), sht.pointer_array(Gs)
    sht.sht_batch_synthesize(B, bp, gp)  # first launch outside the capture
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            sht.sht_batch_synthesize(B, bp, gp, stream=s)
    for rep in range(2):
        for f, l in enumerate(ls):
            betas[f].copy_(torch.from_numpy(inputs.random_beta(l, seed=3000 + 100 * rep + f)))
        g.replay()
        torch.cuda.synchronize()
        assert sht.sht_batch_last_device_status(B) == 0
        for l, beta, G in zip(ls, betas, Gs):
            ref = torch.empty_like(G)
            sht.sht_legendre_synthesize(plans[l], 0, beta, ref)
            torch.cuda.synchronize()
            assert torch.equal(G, ref)
    del g
    B.close()


def test_batch_autotune_keeps_results(sht, plans):
    ls = field_ls(9, 6)
    for l in set(ls):
        plans[l].prepare(2)
    B = sht.Batch([plans[l] for l in ls], 2)
    betas, Gs = fields(ls, 2, 4000)
    bp, gp = sht.pointer_array(betas), sht.pointer_array(Gs)
    cfg = sht.sht_batch_autotune(B, 0, bp, gp, reps=2)
    assert cfg["consumer_warps"] in (8, 12, 16) and 2 <= cfg["nstages"] <= 8
    Gs2 = [torch.full_like(G, float("nan")) for G in Gs]
    sht.sht_batch_synthesize(B, bp, sht.pointer_array(Gs2))
    assert sht.sht_batch_last_device_status(B) == 0
    for l, beta, G in zip(ls, betas, Gs2):
        ref = torch.empty_like(G)
        sht.sht_legendre_synthesize(plans[l], 2, beta, ref)
        torch.cuda.synchronize()
        assert torch.equal(G, ref)
    B.close()


def test_batch_bad_pointer_entry_is_reported(sht, plans):
    """A misaligned output pointer of one field is caught on the device before
    any of that field's pages are issued; the batch works again afterwards."""
    ls = [16, 32, 64]
    B = sht.Batch([plans[l] for l in ls], 0)
    betas, Gs = fields(ls, 0, 5000)
    bad = [betas[0].data_ptr(), betas[1].data_ptr() + 8, betas[2].data_ptr()]
    bp = torch.tensor(bad, dtype=torch.int64, device="cuda")
    sht.sht_batch_synthesize(B, bp, sht.pointer_array(Gs))
    assert sht.sht_batch_last_device_status(B) == 1
    bp = sht.pointer_array(betas)
    sht.sht_batch_synthesize(B, bp, sht.pointer_array(Gs))
    assert sht.sht_batch_last_device_status(B) == 0
    for l, beta, G in zip(ls, betas, Gs):
        assert rel(G, oracle.legendre_synthesis(beta.cpu().numpy(), l)) < TOL[0]
    B.close()


def test_batch_with_degenerate_and_single_fields(sht, plans):
    """Fields of bandlimit 1 and 2 (a handful of coefficients, dense blocks
    only) batched with larger ones, and a batch of a single field."""
    tiny = {l: sht.Plan(l, 1e-12, leaf_cols=4) for l in (1, 2)}
    ls = [1, 64, 2, 4, 1, 128]
    pl = [tiny[l] if l in tiny else plans[l] for l in ls]
    for prec in (0, 3, 1):
        for p in set(pl):
            p.prepare(prec)
        B = sht.Batch(pl, prec)
        betas, Gs = fields(ls, prec, 7000)
        sht.sht_batch_synthesize(B, sht.pointer_array(betas), sht.pointer_array(Gs))
        assert sht.sht_batch_last_device_status(B) == 0
        for l, beta, G in zip(ls, betas, Gs):
            assert rel(G, oracle.legendre_synthesis(beta.cpu().numpy().astype(np.complex128), l)) < TOL[prec], l
        B.close()
    one = sht.Batch([plans[32]], 0)
    betas, Gs = fields([32], 0, 7100)
    sht.sht_batch_synthesize(one, sht.pointer_array(betas), sht.pointer_array(Gs))
    assert sht.sht_batch_last_device_status(one) == 0
    ref = torch.empty_like(Gs[0])
    sht.sht_legendre_synthesize(plans[32], 0, betas[0], ref)
    torch.cuda.synchronize()
    assert torch.equal(ref, Gs[0])
    one.close()


@pytest.mark.parametrize("prec", [0, 2, 1])
def test_batch_grid_equals_per_field_full_transforms(sht, plans, prec):
    """sht_batch_synthesize_grid / sht_batch_analyze_grid (one batched
    Legendre launch with the phase fused, plus each field's FFTs) give each
    field exactly the values of sht_synthesize / sht_analyze, and match the
    oracle's full transforms."""
    ls = field_ls(7, 8)
    for l in set(ls):
        plans[l].prepare(prec)
    B = sht.Batch([plans[l] for l in ls], prec)
    rdt = torch.float32 if prec == 1 else torch.float64
    betas, _ = fields(ls, prec, 9000)
    values = [torch.full((2 * l, 4 * l - 1), float("nan"), dtype=rdt, device="cuda") for l in ls]
    ws = [torch.empty((2 * l, 2 * l), dtype=CDT[prec], device="cuda") for l in ls]
    for _ in range(5):  # more calls than the pointer-table ring has slots
        sht.sht_batch_synthesize_grid(B, betas, values, ws)
    torch.cuda.synchronize()
    assert sht.sht_batch_last_device_status(B) == 0
    for l, beta, v in zip(ls, betas, values):
        ref = torch.full_like(v, float("nan"))
        sht.sht_synthesize(plans[l], prec, beta, ref, torch.empty((2 * l, 2 * l), dtype=CDT[prec], device="cuda"))
        torch.cuda.synchronize()
        assert torch.equal(v, ref), l
    f0 = ls[0]
    fo = oracle.sht_synthesis(betas[0].cpu().numpy().astype(np.complex128), f0)
    assert np.linalg.norm(values[0].cpu().numpy() - fo) / np.linalg.norm(fo) < TOL[prec]
    backs = [torch.full_like(b, float("nan")) for b in betas]
    sht.sht_batch_analyze_grid(B, values, backs, ws)
    torch.cuda.synchronize()
    assert sht.sht_batch_last_device_status(B) == 0
    for l, v, back in zip(ls, values, backs):
        ref = torch.full_like(back, float("nan"))
        sht.sht_analyze(plans[l], prec, v, ref, torch.empty((2 * l, 2 * l), dtype=CDT[prec], device="cuda"))
        torch.cuda.synchronize()
        assert torch.equal(back, ref), l
    for b, back in zip(betas, backs):
        assert rel(back, b) < 2 * TOL[prec]
    B.close()


def test_batch_grid_rejects_bad_pointers(sht, plans):
    ls = [16, 32]
    B = sht.Batch([plans[l] for l in ls], 0)
    betas, _ = fields(ls, 0, 9100)
    values = [torch.empty((2 * l, 4 * l - 1), dtype=torch.float64, device="cuda") for l in ls]
    ws = [torch.empty((2 * l, 2 * l), dtype=torch.complex128, device="cuda") for l in ls]
    with pytest.raises(sht.ShtError) as e:
        sht.sht_batch_synthesize_grid(B, betas, values, [ws[0], ws[1].data_ptr() + 8])
    assert e.value.code == 1
    sht.sht_batch_synthesize_grid(B, betas, values, ws)
    assert sht.sht_batch_last_device_status(B) == 0
    B.close()


@pytest.mark.parametrize("prec", [0, 2, 1])
def test_batched_spellings_match_oracle(sht, plans, prec):
    """sht_synthesize_batched / sht_analyze_batched (a batch built for the
    call, one workspace buffer split per field) against the oracle's full
    transforms of every field, and the same values as the batch object."""
    ls = field_ls(11, 6)
    pl = [plans[l] for l in ls]
    for p in set(pl):
        p.prepare(prec)
    rdt = torch.float32 if prec == 1 else torch.float64
    betas, _ = fields(ls, prec, 9300)
    values = [torch.full((2 * l, 4 * l - 1), float("nan"), dtype=rdt, device="cuda") for l in ls]
    need = sht.sht_batched_workspace_bytes(pl, prec)
    assert need >= sum(sht.sht_workspace_bytes(p, prec) for p in pl)
    ws = torch.empty(need, dtype=torch.uint8, device="cuda")
    sht.sht_synthesize_batched(pl, prec, betas, values, ws)
    for l, beta, v in zip(ls, betas, values):
        fo = oracle.sht_synthesis(beta.cpu().numpy().astype(np.complex128), l)
        assert np.linalg.norm(v.cpu().numpy() - fo) / np.linalg.norm(fo) < TOL[prec], l
    backs = [torch.full_like(b, float("nan")) for b in betas]
    sht.sht_analyze_batched(pl, prec, values, backs, ws)
    for l, v, back in zip(ls, values, backs):
        bo = oracle.sht_analysis(v.cpu().numpy().astype(np.float64), l)
        assert rel(back, bo) < TOL[prec], l
    B = sht.Batch(pl, prec)
    again = [torch.full_like(v, float("nan")) for v in values]
    per = [torch.empty((2 * l, 2 * l), dtype=CDT[prec], device="cuda") for l in ls]
    sht.sht_batch_synthesize_grid(B, betas, again, per)
    torch.cuda.synchronize()
    for v, a in zip(values, again):
        assert torch.equal(v, a)
    B.close()
    st = sht.sht_plan_stats(pl[0])
    assert st == pl[0].stats() and st["l"] == ls[0]


@pytest.mark.parametrize("prec", [0, 2, 3, 1])
def test_fields_sharing_a_plan_run_in_groups(sht, plans, prec):
    """Fields that share a plan run in groups: each op's values are staged
    once and applied to every field of the group.  Nine fields of one plan
    form three groups of three (balanced, at most four per group), a plan
    that appears once stays alone; every field equals its per-field call bit
    for bit in both directions, also after the autotuner has chosen the cap
    on fields per group."""
    pl = [plans[64]] * 9 + [plans[128]]
    ls = [64] * 9 + [128]
    for p in set(pl):
        p.prepare(prec)
    B = sht.Batch(pl, prec)
    assert B.groups(0) == (4, 4)  # three groups of three fields, one of one
    betas, Gs = fields(ls, prec, 9500)
    Gin = [torch.from_numpy(inputs.random_G(l, seed=9600 + f)).to(CDT[prec]).cuda() for f, l in enumerate(ls)]
    backs = [torch.full_like(b, float("nan")) for b in betas]

    def check():
        sht.sht_batch_synthesize(B, sht.pointer_array(betas), sht.pointer_array(Gs))
        sht.sht_batch_analyze(B, sht.pointer_array(Gin), sht.pointer_array(backs))
        assert sht.sht_batch_last_device_status(B) == 0
        for p, beta, G, g, back in zip(pl, betas, Gs, Gin, backs):
            ref = torch.full_like(G, float("nan"))
            sht.sht_legendre_synthesize(p, prec, beta, ref)
            rb = torch.full_like(back, float("nan"))
            sht.sht_legendre_analyze(p, prec, g, rb)
            torch.cuda.synchronize()
            assert torch.equal(G, ref) and torch.equal(back, rb)
        l = ls[0]
        assert rel(Gs[0], oracle.legendre_synthesis(betas[0].cpu().numpy().astype(np.complex128), l)) < TOL[prec]

    check()
    sht.sht_batch_autotune(B, 0, sht.pointer_array(betas), sht.pointer_array(Gs), reps=2)
    assert B.groups(0)[0] in (1, 2, 4)
    check()
    B.close()
