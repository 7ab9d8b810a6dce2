"""The training loss as a torch.autograd.Function (forward and hand-written
backward in the fused tensor-core kernel): gradients against the FP64
analytic gradient of the oracle (itself pinned by finite differences in
test_oracle_train), the chain rule, and an optimisation run through it."""
import numpy as np
import pytest

import oracle
import wost_inputs as wi

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def mods():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_2410_18944_gb300 import api, autograd, build
    build.build()
    return api, autograd


def _setup(api, dim, seed, positive):
    sc = wi.half_disk(48, 12) if dim == 2 else wi.slab_box(2)
    lo, hi = sc.padded_bbox()
    F = api.Field(dim, lo, hi)
    fp = wi.random_field_params(dim, seed, lo, hi, log2T=F.desc.log2_table, w_scale=0.5)
    if positive:
        fp["grid"] = np.abs(fp["grid"]) + 0.05
        fp["W1"], fp["W2"] = np.abs(fp["W1"]), np.abs(fp["W2"])
    fp["grid"] = wi.round_to_fp16(fp["grid"])
    for k in ("W1", "W2", "W3"):
        fp[k] = wi.round_to_bf16(fp[k])
    fp["b3"] = fp["b3"].astype(np.float32).astype(np.float64)
    OF = oracle.Field(oracle.FieldParams(**fp))
    O = oracle.Scene(sc)
    rng = np.random.default_rng(seed)
    pts = []
    while len(pts) < 64:
        p = rng.uniform(*sc.bbox)
        if O.winding(p[None])[0] > 0.5 and O.closest_dirichlet(p[None])[1][0] > 0.05:
            pts.append(p)
    r = oracle.solve(O, oracle.make_params(eps=1e-3, maxsteps=256, seed=3, guided=1), np.array(pts), 0, 1,
                     field=OF, records=True)
    recs = r["records"].astype(np.float32)
    F.set_records(recs)
    tens = [torch.tensor(fp[k], dtype=torch.float32, device="cuda", requires_grad=True)
            for k in ("grid", "W1", "W2", "W3", "b3")]
    return F, OF, recs, tens


@pytest.mark.parametrize("dim", [2, 3])
def test_autograd_matches_fp64_gradient(mods, dim):
    api, ag = mods
    F, OF, recs, tens = _setup(api, dim, 40 + dim, positive=True)
    loss = ag.field_loss(F, *tens)
    loss.backward()
    ol, og, _ = OF.train_loss(recs.astype(np.float64))
    assert loss.item() == pytest.approx(ol, rel=2e-2)
    for name, t, o in zip(["grid", "W1", "W2", "W3", "b3"], tens, og):
        gv = t.grad.double().cpu().numpy().ravel()
        ov = o.ravel()
        cos = gv @ ov / (np.linalg.norm(gv) * np.linalg.norm(ov) + 1e-300)
        rel = np.linalg.norm(gv - ov) / (np.linalg.norm(ov) + 1e-300)
        # BF16 operands / FP32 accumulation against FP64: rel-L2 < 2e-2,
        # cosine > 0.999
        assert cos > 0.999 and rel < 2e-2, (name, cos, rel)


def test_autograd_chain_rule_and_partial_inputs(mods):
    api, ag = mods
    F, OF, recs, tens = _setup(api, 2, 7, positive=False)
    g1 = torch.autograd.grad(ag.field_loss(F, *tens), tens)
    g3 = torch.autograd.grad(3.0 * ag.field_loss(F, *tens) + 1.0, tens)
    for a, b in zip(g1, g3):
        assert torch.allclose(3.0 * a, b, rtol=1e-4, atol=1e-9)
    # gradients only for some inputs
    grid = tens[0].detach().requires_grad_(True)
    rest = [t.detach() for t in tens[1:]]
    (gg,) = torch.autograd.grad(ag.field_loss(F, grid, *rest), [grid])
    assert torch.allclose(gg, g1[0], rtol=1e-4, atol=1e-9)


def test_optimisation_through_the_function_lowers_the_loss(mods):
    api, ag = mods
    F, OF, recs, tens = _setup(api, 2, 11, positive=False)
    opt = torch.optim.Adam(tens, lr=3e-3)
    losses = []
    for _ in range(12):
        opt.zero_grad()
        loss = ag.field_loss(F, *tens)
        loss.backward()
        opt.step()
        losses.append(loss.item())
    assert np.all(np.isfinite(losses))
    assert losses[-1] < losses[0]


@pytest.mark.parametrize("dim", [2, 3])
def test_forward_computes_the_loss_only(mods, dim):
    # forward runs the kernel's loss-only mode: the same loss as the full
    # gradient pass, also under no_grad, and it leaves the field's gradient
    # buffers alone (backward computes them)
    api, ag = mods
    F, OF, recs, tens = _setup(api, dim, 50 + dim, positive=False)
    with torch.no_grad():
        l0 = ag.field_loss(F, *tens)
    assert l0.device.type == "cuda" and not l0.requires_grad
    lg, _ = F.train_grad()
    assert float(l0) == pytest.approx(lg, rel=1e-6)
    loss = ag.field_loss(F, *tens)
    assert float(loss.detach()) == pytest.approx(lg, rel=1e-6)
    loss.backward()
    g_ref = F.train_grad()[1]
    for t, k in zip(tens, ("grid", "W1", "W2", "W3", "b3")):
        assert np.allclose(t.grad.cpu().numpy(), g_ref[k], rtol=1e-5, atol=1e-7 * np.abs(g_ref[k]).max())
