"""FP64 reference of the learned warm start's network: forward pass, loss and
the gradient by hand-written backpropagation.

TEST INFRASTRUCTURE ONLY (see oracle/__init__.py).  Plain numpy, direct
transforms from oracle.sht.  Used to check the CUDA kernels' loss and
gradients; pinned itself by finite differences.

Network (parameters one flat vector, same order as the library):
  inputs per pixel: c0 = (1-m) d / sigma_d, c1 = (1-m)(log sigma^2 - mu)/s,
  c2 = m  (sigma_d, mu, s over observed pixels);
  per-ring circular convolutions, taps k = 0..K-1 at offset k - K//2:
  h1 = relu(W1*c + b1), h2 = relu(W2*h1 + b2), r = W3*h2 + b3;
  t0 = (1-m) d + sigma_d r;  a = Omega Y^T t0;
  features per l: (l/lmax, log10 C/10, log10(P_d/C)/5, log10(alpha Omega/C)/5)
  (clipped to [-4, 4]; P_d = power of Omega Y^T((1-m) d));
  q_l = sigmoid(V3 relu(V2 relu(V1 f + c1) + c2) + c3);  a0 = q_l a;
  loss = sum w |a0 - a*|^2 / sum w |a*|^2.
"""
import numpy as np

from . import sht


def layout(H, K, Hm):
    sizes = [("W1", (H, 3, K)), ("b1", (H,)), ("W2", (H, H, K)), ("b2", (H,)),
             ("W3", (1, H, K)), ("b3", (1,)), ("V1", (Hm, 4)), ("c1", (Hm,)),
             ("V2", (Hm, Hm)), ("c2", (Hm,)), ("V3", (1, Hm)), ("c3", (1,))]
    out, o = {}, 0
    for name, shp in sizes:
        n = int(np.prod(shp))
        out[name] = (o, shp)
        o += n
    return out, o


def unpack(theta, H, K, Hm):
    lay, _ = layout(H, K, Hm)
    return {k: theta[o:o + int(np.prod(s))].reshape(s) for k, (o, s) in lay.items()}


def rings(nside):
    out = []
    for r in range(1, 4 * nside):
        f, n, _, _, _ = sht.ring_info(nside, r)
        out.append((f, n))
    return out


def conv(x, W, b, rs):
    """x: (cin, npix) -> (cout, npix), circular along each ring."""
    cout, cin, K = W.shape
    h = K // 2
    y = np.zeros((cout, x.shape[1]))
    for f, n in rs:
        seg = x[:, f:f + n]
        acc = np.tile(b[:, None], (1, n)).astype(np.float64)
        for k in range(K):
            sh = np.roll(seg, -(k - h), axis=1)      # sh[:, j] = seg[:, j + k - h]
            acc += W[:, :, k] @ sh
        y[:, f:f + n] = acc
    return y


def conv_back(g, x, W, rs):
    """Given g = dL/dy, return dL/dx, dL/dW, dL/db."""
    cout, cin, K = W.shape
    h = K // 2
    gx = np.zeros_like(x)
    gW = np.zeros_like(W)
    gb = g.sum(axis=1)
    for f, n in rs:
        gs = g[:, f:f + n]
        seg = x[:, f:f + n]
        for k in range(K):
            sh = np.roll(seg, -(k - h), axis=1)
            gW[:, :, k] += gs @ sh.T
            # y[:, j] uses x[:, j + k - h]: scatter back
            gx[:, f:f + n] += np.roll(W[:, :, k].T @ gs, (k - h), axis=1)
    return gx, gW, gb


def forward(theta, H, K, Hm, nside, lmax, cl, noise_var, mask, d, alpha=None):
    p = unpack(np.asarray(theta, dtype=np.float64), H, K, Hm)
    om = 4 * np.pi / sht.npix(nside)
    obs = ~mask
    a_ = float(np.min(noise_var[obs])) if alpha is None else alpha
    dm = np.where(mask, 0.0, d)
    sig = np.sqrt(np.sum(dm[obs] ** 2) / obs.sum())
    lg = np.log(noise_var[obs])
    mu = lg.mean()
    sd = np.sqrt(max(np.mean(lg ** 2) - mu * mu, 0.0))
    sd = sd if sd > 1e-12 else 1.0
    c = np.zeros((3, len(d)))
    c[0] = np.where(mask, 0.0, d / sig)
    c[1] = np.where(mask, 0.0, (np.log(noise_var) - mu) / sd)
    c[2] = mask.astype(float)
    rs = rings(nside)
    z1 = conv(c, p["W1"], p["b1"], rs)
    h1 = np.maximum(z1, 0)
    z2 = conv(h1, p["W2"], p["b2"], rs)
    h2 = np.maximum(z2, 0)
    r = conv(h2, p["W3"], p["b3"], rs)[0]
    t0 = dm + sig * r
    a = sht.map2alm(t0, nside, lmax)
    ad = sht.map2alm(dm, nside, lmax)
    ls, ms = sht.lm_arrays(lmax)
    w = np.where(ms == 0, 1.0, 2.0)
    pd = np.zeros(lmax + 1)
    np.add.at(pd, ls, w * np.abs(ad) ** 2)
    pd /= (2 * np.arange(lmax + 1) + 1)
    cc = np.asarray(cl, dtype=np.float64) + 1e-30
    ell = np.arange(lmax + 1)
    F = np.stack([ell / lmax,
                  np.clip(np.log10(cc) / 10, -4, 4),
                  np.clip(np.log10((pd + 1e-30) / cc) / 5, -4, 4),
                  np.clip(np.log10(a_ * om / cc) / 5, -4, 4)], axis=1)
    u1 = F @ p["V1"].T + p["c1"]
    m1 = np.maximum(u1, 0)
    u2 = m1 @ p["V2"].T + p["c2"]
    m2 = np.maximum(u2, 0)
    zz = (m2 @ p["V3"].T)[:, 0] + p["c3"][0]
    q = 1 / (1 + np.exp(-zz))
    a0 = q[ls] * a
    return dict(p=p, c=c, h1=h1, h2=h2, t0=t0, a=a, a0=a0, F=F, m1=m1, m2=m2, q=q,
                sig=sig, rs=rs, om=om, ls=ls, w=w)


def loss_grad(theta, H, K, Hm, nside, lmax, cl, noise_var, mask, d, target):
    """Loss and its gradient (flat vector) w.r.t. theta."""
    st = forward(theta, H, K, Hm, nside, lmax, cl, noise_var, mask, d)
    p, w, ls = st["p"], st["w"], st["ls"]
    diff = st["a0"] - target
    norm = np.sum(w * np.abs(target) ** 2)
    loss = np.sum(w * np.abs(diff) ** 2) / norm
    # dL/dq_l
    dq = np.zeros(lmax + 1)
    np.add.at(dq, ls, w * 2 * (diff.real * st["a"].real + diff.imag * st["a"].imag) / norm)
    q = st["q"]
    dz = dq * q * (1 - q)
    g = {}
    g["c3"] = np.array([dz.sum()])
    g["V3"] = (dz[:, None] * st["m2"]).sum(axis=0)[None, :]
    d2 = (dz[:, None] * p["V3"]) * (st["m2"] > 0)
    g["c2"] = d2.sum(axis=0)
    g["V2"] = d2.T @ st["m1"]
    d1 = (d2 @ p["V2"]) * (st["m1"] > 0)
    g["c1"] = d1.sum(axis=0)
    g["V1"] = d1.T @ st["F"]
    # a0 = q a, a = Omega Y^T t0 -> dL/dt0 = Omega Y (2 q diff / norm)
    b = 2 * q[ls] * diff / norm
    gt0 = st["om"] * sht.alm2map(b, nside, lmax)
    gr = st["sig"] * gt0
    g3 = gr[None, :]
    gh2, g["W3"], g["b3"] = conv_back(g3, st["h2"], p["W3"], st["rs"])
    gz2 = gh2 * (st["h2"] > 0)
    gh1, g["W2"], g["b2"] = conv_back(gz2, st["h1"], p["W2"], st["rs"])
    gz1 = gh1 * (st["h1"] > 0)
    _, g["W1"], g["b1"] = conv_back(gz1, st["c"], p["W1"], st["rs"])
    lay, n = layout(H, K, Hm)
    flat = np.zeros(n)
    for k, (o, s) in lay.items():
        flat[o:o + int(np.prod(s))] = np.asarray(g[k]).reshape(-1)
    return loss, flat
