"""Training-side kernels against the FP64 oracles: the fused Adam step, raw-parameter rendering
(log-scales and opacity logits activated by the kernels, gradients chained through them) and
densification on raw parameters."""
import numpy as np
import pytest

from oracle import densify as OD
from oracle import oracle as O
from oracle import train as OT
from paper_2410_20686_gb300 import scenes as S
from tests.helpers import EPS_CLAMP, EPS_SKIP, EPS_TERM, IMG_TOL, assert_grads_close, compare_image, oracle_settings

pytestmark = pytest.mark.gpu
NAMES = ("means", "scales", "quats", "opacity", "sh")


@pytest.mark.parametrize("n,offset", [(1001, 0), (4096, 0), (777, 1)])
def test_adam_matches_the_oracle_over_five_steps(n, offset):
    import torch
    from paper_2410_20686_gb300.optim import GaussianAdam
    rng = np.random.default_rng(n + offset)
    shapes = [(n, 3), (n, 3), (n, 4), (n,), (n, 16, 3)]
    host = [rng.normal(size=s).astype(np.float32) for s in shapes]
    # offset > 0 places the tensors one float past a 16-byte boundary (the scalar path)
    dev = [torch.from_numpy(np.concatenate([np.zeros(offset, np.float32), h.ravel()])).cuda()[offset:].view(h.shape)
           for h in host]
    opt = GaussianAdam(dev, scene_extent=3.0)
    ref = [(h.astype(np.float64), np.zeros(h.shape), np.zeros(h.shape)) for h in host]
    lr = [np.float64(opt.lr[k]) for k in ("means", "scales", "quats", "opacity")]
    sh_lr = np.where(np.arange(48).reshape(16, 3) < 3, opt.lr["sh_dc"], opt.lr["sh_rest"])[None]
    lr.append(sh_lr)
    for step in range(1, 6):
        grads = [rng.normal(scale=10.0 ** rng.uniform(-4, 1), size=s).astype(np.float32) for s in shapes]
        opt.step([torch.from_numpy(g).cuda() for g in grads])
        ref = [OT.adam(p, g, m, v, step, l, eps=opt.eps) for (p, m, v), g, l in zip(ref, grads, lr)]
    torch.cuda.synchronize()
    # float32 moments carry rounding of the largest term that entered them (the gradient scales of
    # the steps differ by up to 1e5, so m can cancel); an update is at most about lr per step, and
    # its error follows from the moments' error relative to the element's own gradient history
    for k, (p, m, v) in enumerate(ref):
        pg = dev[k].cpu().numpy()
        np.testing.assert_allclose(opt.m[k].cpu().numpy(), m, rtol=1e-5, atol=1e-6 * np.abs(m).max())
        np.testing.assert_allclose(opt.v[k].cpu().numpy(), v, rtol=1e-5, atol=1e-6 * np.abs(v).max())
        # each of the 5 steps also rounds p itself to float32 (half an ulp of |p|)
        d_ref = p - host[k]
        bound = 1e-4 * np.abs(d_ref) + 1e-4 * float(np.max(lr[k])) + 5 * np.spacing(np.abs(host[k]) + 1e-3)
        worst = np.max(np.abs((pg - host[k]) - d_ref) / bound)
        assert worst <= 1.0, f"parameter group {k}: update error {worst:.2f} x the bound"


def _raw_scene():
    sc = S.random_scene(400, 256, 128, seed=21, sh_degree=3, radius=(1.5, 5.0), log_scale=(-3.5, 0.5))
    log_s = np.log(sc.scales).astype(np.float32)
    logit = np.log(sc.opacity / (1.0 - sc.opacity)).astype(np.float32)
    s, o = OT.activate(log_s, logit)  # the oracle's scene: FP64 activations of the raw float32 values
    return sc, log_s, logit, O.Params(sc.means, s, sc.quats, o, sc.sh)


def test_raw_parameters_render_and_differentiate_like_the_activated_oracle():
    import torch
    from paper_2410_20686_gb300.rasterizer import Rasterizer, RenderSettings
    sc, log_s, logit, p = _raw_scene()
    rs = RenderSettings(sh_degree=3, raw_params=True)
    st = oracle_settings(rs)
    v = sc.views[0]
    col, _, _, margins = O.render(p, v, st)
    amb = O.ambiguous(margins, EPS_SKIP, EPS_TERM, EPS_CLAMP)
    w = np.random.default_rng(2).normal(size=(3, v.height, v.width)) * (~amb)[None]
    params = [torch.tensor(a, device="cuda") for a in (sc.means, log_s, sc.quats, logit, sc.sh)]
    rast = Rasterizer()
    imgs, _ = rast.forward(*params, [v], rs, want_T=False)
    g = rast.backward([torch.tensor(w, dtype=torch.float32, device="cuda")])
    torch.cuda.synchronize()
    assert rast.status() == 0
    compare_image(imgs[0].cpu().numpy().astype(np.float64), col, margins, tol=IMG_TOL)
    ref = O.backward(p, v, st, w)
    ref["scales"], ref["opacity"] = OT.chain(log_s, logit, ref["scales"], ref["opacity"])
    assert_grads_close({k: g[k].cpu().numpy().astype(np.float64) for k in NAMES}, ref, NAMES)


def test_densification_on_raw_parameters_matches_the_oracle():
    import torch
    from paper_2410_20686_gb300.densify import DensifyParams, DensifyStats, apply, select
    rng = np.random.default_rng(9)
    n = 50_000
    count = rng.integers(0, 5, n).astype(np.uint32)
    elev = (rng.uniform(0, 1, n) * count).astype(np.float32)
    grad = (rng.uniform(0, 2e-4, n) * count).astype(np.float32)
    log_s = np.log(rng.uniform(2e-4, 8e-3, (n, 3))).astype(np.float32)
    logit = rng.normal(-4.0, 1.5, n).astype(np.float32)
    prm = DensifyParams(scene_extent=2.0, max_scale=6e-3, raw_params=True)
    st = DensifyStats(n)
    st.grad.copy_(torch.from_numpy(grad))
    st.elev.copy_(torch.from_numpy(elev))
    st.count.copy_(torch.from_numpy(count.astype(np.int32)))
    ls, lo = torch.from_numpy(log_s).cuda(), torch.from_numpy(logit).cuda()
    act = select(st, ls, lo, prm).cpu().numpy()
    ref = OD.select(grad, elev, count, log_s, logit, OD.DensifyParams(**prm.__dict__))
    np.testing.assert_array_equal(act, ref)
    assert all(np.count_nonzero(ref == a) > 100 for a in (OD.KEEP, OD.CLONE, OD.SPLIT, OD.PRUNE))
    means = rng.normal(size=(n, 3)).astype(np.float32)
    quats = rng.normal(size=(n, 4)).astype(np.float32)
    sh = rng.normal(size=(n, 4, 3)).astype(np.float32)
    noise = rng.normal(size=(n, 2, 3)).astype(np.float32)
    t = [torch.from_numpy(a).cuda() for a in (means, log_s, quats, logit, sh)]
    out = apply(*t, torch.from_numpy(act).cuda(), torch.from_numpy(noise).cuda(), raw_params=True)
    want = OD.apply(means, log_s, quats, logit, sh, act, noise, raw_params=True)
    for a, b in zip(out, want):
        a = a.cpu().numpy()
        assert a.shape == b.shape
        np.testing.assert_allclose(a, b, rtol=2e-6, atol=2e-6)
