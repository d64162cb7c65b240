"""FP64 reference of the learned near-field preconditioner network (test infrastructure).

Not in the paper: the paper's preconditioner is the diagonal of L_s, and it
notes that off-diagonal entries may augment it (Sec. III-A-2).  The learned
form used by the library is

    M = D^{-1} (I + C),   C supported on the near-region graph (and its diagonal),

with D the per-basis static self block.  A message-passing network over the
near graph maps node and edge features to the entries of C:

    h0      = relu(A0 x_m + a0)
    p_n     = B_l h_{l-1,n}
    q_mn    = relu(p_n + C_l e_mn + c_l)                 (edges n -> m, n != m)
    s_m     = (1 / deg_m) sum_n q_mn
    h_l     = relu(D_l h_{l-1,m} + s_m + d_l),           l = 1..L
    o_mn    = E (h_{L,m} * h_{L,n}) + F e_mn + f          (edge outputs, K reals)
    g_m     = G h_{L,m} + g                               (diagonal outputs, K reals)

K = 2 (one complex entry, EFIE) or 8 (a 2x2 complex block, two-region form,
row-major (E,J), (E,M), (H,J), (H,M), real then imaginary).  Training
minimises the probe loss

    L = (1/P) sum_p |M y_p - z_p|^2 / |z_p|^2,   y_p = A z_p,

which is quadratic in C, so A is only needed through the fixed pairs (z, y).

This module computes the forward pass, the loss and all parameter gradients
in float64 by explicit backpropagation; tests compare the CUDA kernels with it
and pin it with central finite differences.
"""

import numpy as np

PARAM_ORDER = ["A0", "a0"] + [f"{n}{l}" for l in range(1, 5) for n in ("B", "C", "c", "D", "d")] + \
    ["E", "F", "f", "G", "g"]


def param_shapes(width=64, layers=4, nin=8, nedge=8, K=2):
    s = {"A0": (width, nin), "a0": (width,)}
    for l in range(1, layers + 1):
        s[f"B{l}"] = (width, width)
        s[f"C{l}"] = (width, nedge)
        s[f"c{l}"] = (width,)
        s[f"D{l}"] = (width, width)
        s[f"d{l}"] = (width,)
    s.update({"E": (K, width), "F": (K, nedge), "f": (K,), "G": (K, width), "g": (K,)})
    return s


def relu(v):
    return np.maximum(v, 0.0)


def forward(params, x, e, rows, cols, layers=4):
    """x [N, nin], e [nnz, nedge] (per stored near pair, diagonal rows included but skipped).

    Returns (o [nnz, K] with zero rows on the diagonal, g [N, K], cache)."""
    N = len(x)
    off = rows != cols
    deg = np.maximum(np.bincount(rows[off], minlength=N), 1).astype(np.float64)
    h = [relu(x @ params["A0"].T + params["a0"])]
    cache = {"deg": deg, "off": off, "w": []}
    for l in range(1, layers + 1):
        hp = h[-1]
        p = hp @ params[f"B{l}"].T
        w = p[cols] + e @ params[f"C{l}"].T + params[f"c{l}"]
        q = relu(w) * off[:, None]
        s = np.zeros_like(hp)
        np.add.at(s, rows, q)
        s /= deg[:, None]
        u = hp @ params[f"D{l}"].T + s + params[f"d{l}"]
        h.append(relu(u))
        cache["w"].append(w)
    hL = h[-1]
    o = (hL[rows] * hL[cols]) @ params["E"].T + e @ params["F"].T + params["f"]
    o = o * off[:, None]
    g = hL @ params["G"].T + params["g"]
    cache["h"] = h
    return o, g, cache


def to_complex_blocks(o, g, K):
    """Edge and diagonal outputs as complex entries: [..] (K=2) or [.., 2, 2] (K=8)."""
    if K == 2:
        return o[:, 0] + 1j * o[:, 1], g[:, 0] + 1j * g[:, 1]
    oc = (o[:, 0:4] + 1j * o[:, 4:8]).reshape(-1, 2, 2)
    gc = (g[:, 0:4] + 1j * g[:, 4:8]).reshape(-1, 2, 2)
    return oc, gc


def apply_precond(dinv, oc, gc, rows, cols, v, K):
    """z = D^{-1} (v + C v); dinv [N] (K=2) or [N,2,2] (K=8); v [nunk] with nunk = N or 2N."""
    N = len(dinv)
    if K == 2:
        t = v + gc * v
        np.add.at(t, rows, oc * v[cols])
        return dinv * t
    V = np.stack([v[:N], v[N:]], axis=1)                       # [N, 2]
    T = V + np.einsum("nab,nb->na", gc, V)
    np.add.at(T, rows, np.einsum("eab,eb->ea", oc, V[cols]))
    Z = np.einsum("nab,nb->na", dinv, T)
    return np.r_[Z[:, 0], Z[:, 1]]


def loss_and_grads(params, x, e, rows, cols, dinv, Y, Zp, K, layers=4):
    """Probe loss and gradients of every parameter (dict), float64."""
    o, g, cache = forward(params, x, e, rows, cols, layers)
    oc, gc = to_complex_blocks(o, g, K)
    N = len(x)
    P = len(Y)
    L = 0.0
    G_e = np.zeros((len(rows), K))
    G_n = np.zeros((N, K))
    for p in range(P):
        y, z = Y[p], Zp[p]
        wgt = 1.0 / (P * np.vdot(z, z).real)
        r = apply_precond(dinv, oc, gc, rows, cols, y, K) - z
        L += wgt * np.vdot(r, r).real
        if K == 2:
            rd = np.conj(r) * dinv                        # conj(r_m) dinv_m
            ge = rd[rows] * y[cols]
            gn = rd * y
            G_e += 2 * wgt * np.stack([ge.real, -ge.imag], 1)
            G_n += 2 * wgt * np.stack([gn.real, -gn.imag], 1)
        else:
            R = np.stack([r[:N], r[N:]], 1)
            Vy = np.stack([y[:N], y[N:]], 1)
            RD = np.einsum("ng,nga->na", np.conj(R), dinv)   # sum_g conj(r_g) dinv[g][a]
            ge = RD[rows][:, :, None] * Vy[cols][:, None, :]  # [E, a, b]
            gn = RD[:, :, None] * Vy[:, None, :]
            G_e += 2 * wgt * np.concatenate([ge.real.reshape(-1, 4), -ge.imag.reshape(-1, 4)], 1)
            G_n += 2 * wgt * np.concatenate([gn.real.reshape(-1, 4), -gn.imag.reshape(-1, 4)], 1)
    off = cache["off"]
    G_e = G_e * off[:, None]
    grads = {k: np.zeros_like(v) for k, v in params.items()}
    h = cache["h"]
    hL = h[-1]
    prod = hL[rows] * hL[cols]
    grads["E"] = G_e.T @ prod
    grads["F"] = G_e.T @ e
    grads["f"] = G_e.sum(0)
    grads["G"] = G_n.T @ hL
    grads["g"] = G_n.sum(0)
    dh = G_n @ params["G"]
    dprod = G_e @ params["E"]
    np.add.at(dh, rows, dprod * hL[cols])
    np.add.at(dh, cols, dprod * hL[rows])
    deg = cache["deg"]
    for l in range(layers, 0, -1):
        hp = h[l - 1]
        du = dh * (h[l] > 0)
        grads[f"D{l}"] = du.T @ hp
        grads[f"d{l}"] = du.sum(0)
        dhp = du @ params[f"D{l}"]
        ds = du / deg[:, None]
        w = cache["w"][l - 1]
        dw = ds[rows] * (w > 0) * off[:, None]
        grads[f"C{l}"] = dw.T @ e
        grads[f"c{l}"] = dw.sum(0)
        dp = np.zeros_like(hp)
        np.add.at(dp, cols, dw)
        grads[f"B{l}"] = dp.T @ hp
        dhp += dp @ params[f"B{l}"]
        dh = dhp
    du0 = dh * (h[0] > 0)
    grads["A0"] = du0.T @ x
    grads["a0"] = du0.sum(0)
    return L, grads


def init_params(seed, width=64, layers=4, nin=8, nedge=8, K=2):
    """He-style initialisation; output layers start at zero so C = 0 (plain preconditioner)."""
    rng = np.random.default_rng(seed)
    out = {}
    for k, shp in param_shapes(width, layers, nin, nedge, K).items():
        if len(shp) == 2 and k not in ("E", "F", "G"):
            out[k] = rng.standard_normal(shp) * np.sqrt(2.0 / shp[1])
        else:
            out[k] = np.zeros(shp)
    return out
