"""Learned troubled-cell selector: training samples from plain-method
trajectories, training with the library's FP32 network kernels
(cgks_mlp_*), thresholds, and the parameter file.

A sample is one cell at one step: its 16 features (cgks_selector_features)
of the state U^n and the label "skippable": the plain method's GENO weights
of that step's first stage, from the same U^n, are all >= 1 - 1e-3, or the
cell's stencil varies by less than 1e-6 of its scale (every feature below
1e-6), where no choice of weights moves its reconstruction by more than
that.  (GENO's absolute epsilon turns variations of order 1e-7, invisible in
FP32 features, into weights below 1; such cells would otherwise be troubled
cells with all-zero features.)  Trajectories are seeded four-quadrant
Riemann problems (outflow boundaries), isentropic vortices, shock-vortex
interactions (Mach 1.1-3, vortex strength 1-5, inflow / outflow / slip
walls) and smooth random
3-D periodic flows (synth.random_smooth_3d), advanced by the plain method
(FP64, no selector).

    python -m paper_2508_08965_gb300.selector --out selector_params.npz
"""
import argparse
import os

import numpy as np

from .binding import Mesh, SEL_NPARAM, mlp_adam, mlp_logits, mlp_loss_grad

HERE = os.path.dirname(os.path.abspath(__file__))
PARAMS = os.path.join(HERE, "selector_params.npz")
CHI_SKIP = 1.0 - 1e-3
TINY = 1e-6
NF, H = 16, 32


def init_params(seed):
    """He-uniform weights (bound sqrt(6 / fan_in)), zero biases."""
    rng = np.random.default_rng(seed)
    out = []
    for fan_in, size in ((NF, H * NF), (0, H), (H, H * H), (0, H), (H, H * H), (0, H), (H, H), (0, 1)):
        out.append(rng.uniform(-np.sqrt(6.0 / fan_in), np.sqrt(6.0 / fan_in), size) if fan_in else np.zeros(size))
    p = np.concatenate(out).astype(np.float32)
    assert p.size == SEL_NPARAM
    return p


def trajectory_samples(mesh, steps):
    """(features, labels) of every cell at each of `steps` steps of a mesh
    advanced by the plain method; torch CUDA tensors."""
    import torch
    X, Y = [], []
    chi = torch.empty((mesh.nv, mesh.ncell), dtype=torch.float64, device="cuda")
    for _ in range(steps):
        f = mesh.selector_features()
        X.append(f)
        mesh.step(1)
        mesh.chi(out=chi)
        Y.append(((chi.min(dim=0).values >= CHI_SKIP) | (f.amax(dim=1) < TINY)).to(torch.float32))
    return torch.cat(X), torch.cat(Y)


def riemann_mesh(seed, n):
    import synth
    states = synth.riemann4_params(seed)
    m = Mesh(2, (n, n), lo=(0.0, 0.0), hi=(1.0, 1.0), bc=[1, 1, 1, 1], tau_mode=1)
    m.init(lambda x, y: synth.riemann4_2d(x, y, states))
    return m


def vortex_mesh(seed, n):
    import synth
    rng = np.random.default_rng(seed)
    eps, c = float(rng.uniform(1.0, 5.0)), tuple(float(x) for x in rng.uniform(2.0, 8.0, 2))
    m = Mesh(2, (n, n), lo=(0.0, 0.0), hi=(10.0, 10.0))
    m.init(lambda x, y: synth.isentropic_vortex_2d(x, y, eps=eps, center=c))
    return m


def shock_vortex_mesh(seed, n):
    """[0, 2] x [0, 1] at 2n x n cells (square cells); shock Mach number in
    [1.1, 3] and vortex strength in [1, 5] drawn by seed."""
    import synth
    mach, eps = synth.shock_vortex_params(seed)
    m = Mesh(2, (2 * n, n), lo=(0.0, 0.0), hi=(2.0, 1.0), bc=[4, 1, 2, 2],
             bc_state=[synth.shock_vortex_inflow(mach)], tau_mode=1)
    m.init(lambda x, y: synth.shock_vortex_2d(x, y, mach, eps))
    return m


def smooth3d_mesh(seed, n):
    import synth
    m = Mesh(3, (n, n, n), lo=(0.0, 0.0, 0.0), hi=(2 * np.pi,) * 3, mu=1e-3, prandtl=0.72, tau_mode=2)
    m.init(lambda x, y, z: synth.random_smooth_3d(x, y, z, seed))
    return m


def build_dataset(riemann_seeds, vortex_seeds, n=256, steps=24, stride=1, smooth3d_seeds=(), n3=32,
                  shock_vortex_seeds=(), shock_vortex_steps=None):
    """Samples of the trajectories; Riemann draws the plain method cannot
    advance are left out (returned as `failed`).  Shock-vortex meshes are
    n x n/2 (the cell size of an n^2 Riemann mesh) and run for
    shock_vortex_steps (default: steps), long enough for the vortex to
    cross the shock."""
    import torch
    from .binding import CgksError
    X, Y, failed = [], [], []
    for kind, seeds in (("riemann", riemann_seeds), ("vortex", vortex_seeds), ("smooth3d", smooth3d_seeds),
                        ("shockvortex", shock_vortex_seeds)):
        for s in seeds:
            nst = steps
            if kind == "riemann":
                m = riemann_mesh(s, n)
            elif kind == "vortex":
                m = vortex_mesh(s, n)
            elif kind == "shockvortex":
                m = shock_vortex_mesh(s, n // 2)
                nst = shock_vortex_steps or steps
            else:
                m = smooth3d_mesh(s, n3)
            try:
                x, y = trajectory_samples(m, nst)
            except CgksError:
                failed.append((kind, s))
                continue
            finally:
                m.close()
            X.append(x[::stride])
            Y.append(y[::stride])
    return torch.cat(X), torch.cat(Y), failed


def train(X, y, epochs=8, batch=16384, lr=3e-3, w_troubled=8.0, seed=0):
    """Adam on the weighted cross-entropy (troubled cells weigh w_troubled:
    a wrong skip costs accuracy, a wrong refusal only time).  Every forward
    and backward pass runs in the library's kernels.  Returns the parameters
    (numpy float32) and the loss of each epoch."""
    import torch
    p = torch.tensor(init_params(seed), device="cuda")
    g = torch.zeros_like(p)
    m = torch.zeros_like(p)
    v = torch.zeros_like(p)
    w = torch.where(y > 0.5, torch.ones_like(y), torch.full_like(y, w_troubled))
    gen = torch.Generator(device="cuda")
    gen.manual_seed(seed)
    n = X.shape[0]
    step, hist = 0, []
    for _ in range(epochs):
        perm = torch.randperm(n, generator=gen, device="cuda")
        tot, cnt = 0.0, 0
        for b0 in range(0, n, batch):
            idx = perm[b0:b0 + batch]
            loss = mlp_loss_grad(p, X[idx].contiguous(), y[idx].contiguous(), w[idx].contiguous(), g)
            step += 1
            mlp_adam(p, g, m, v, step, lr)
            tot += loss * idx.numel()
            cnt += idx.numel()
        hist.append(tot / cnt)
    torch.cuda.synchronize()
    return p.cpu().numpy(), hist


def thresholds(params, X, y, max_false_skip=1e-3, margin=0.5):
    """thr_skip: the smallest logit such that at most max_false_skip of the
    troubled cells (y = 0) of (X, y) reach it, raised by `margin` to cover the
    BF16 rounding of the fused inference; thr_lo = thr_skip - 4."""
    import torch
    z = mlp_logits(torch.tensor(params, device="cuda"), X)
    bad = z[y < 0.5]
    if bad.numel() == 0:
        thr = float(z.min()) - margin
    else:
        k = int(np.floor(max_false_skip * bad.numel()))
        srt = torch.sort(bad, descending=True).values
        thr = float(srt[min(k, srt.numel() - 1)]) + margin
    return thr, thr - 4.0


def load(path=PARAMS):
    d = np.load(path)
    return d["params"].astype(np.float32), float(d["thr_skip"]), float(d["thr_lo"])


def main():
    import torch
    ap = argparse.ArgumentParser()
    ap.add_argument("--out", default=PARAMS)
    ap.add_argument("--n", type=int, default=256)
    ap.add_argument("--steps", type=int, default=24)
    ap.add_argument("--riemann", type=int, default=24)
    ap.add_argument("--vortex", type=int, default=8)
    ap.add_argument("--epochs", type=int, default=8)
    ap.add_argument("--stride", type=int, default=4)
    ap.add_argument("--smooth3d", type=int, default=8)
    ap.add_argument("--shock-vortex", type=int, default=8)
    ap.add_argument("--shock-vortex-steps", type=int, default=192)
    args = ap.parse_args()
    train_r = list(range(0, args.riemann))
    train_v = list(range(1000, 1000 + args.vortex))
    train_s = list(range(2000, 2000 + args.smooth3d))
    train_k = list(range(3000, 3000 + args.shock_vortex))
    X, y, failed = build_dataset(train_r, train_v, args.n, args.steps, args.stride, train_s,
                                 shock_vortex_seeds=train_k, shock_vortex_steps=args.shock_vortex_steps)
    Xv, yv, failed_v = build_dataset(list(range(5000, 5000 + args.riemann // 4)), [6000, 6001], args.n, args.steps,
                                     args.stride, [7000, 7001], shock_vortex_seeds=[8000, 8001],
                                     shock_vortex_steps=args.shock_vortex_steps)
    params, hist = train(X, y, epochs=args.epochs)
    thr, lo = thresholds(params, Xv, yv)
    z = mlp_logits(torch.tensor(params, device="cuda"), Xv)
    skip = (z >= thr)
    info = {
        "samples": int(X.shape[0]), "skippable_fraction": float(y.mean()), "loss_per_epoch": hist,
        "val_skip_rate": float(skip.float().mean()),
        "val_false_skip_rate": float((skip & (yv < 0.5)).float().sum() / max(1, int((yv < 0.5).sum()))),
        "failed_draws": failed + failed_v,
    }
    np.savez(args.out, params=params, thr_skip=thr, thr_lo=lo, info=repr(info))
    print(info)


if __name__ == "__main__":
    main()
