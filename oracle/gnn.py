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


# ------------------------------------------------------------------ inputs of the network

def _wavenumbers(freq, eps_out, eps_in, mu_in):
    from .constants import C0
    k_out = 2.0 * np.pi * freq * np.sqrt(eps_out) / C0
    contrast = 1.0 if eps_in is None else np.sqrt(eps_in * mu_in / eps_out)
    return k_out, contrast


def features(prob, freq, eps_out=1.0, eps_in=None, mu_in=1.0):
    """Node features x [N, 8] and edge features e [nnz, 8] on the near graph (caller order).

    With h_bar the geometric mean of the grid spacings and k the exterior
    wavenumber, every feature is dimensionless:

      node m: l_m/h_bar, A+_m/h_bar^2, A-_m/h_bar^2, the offset of the basis
              centre from the stencil's central node in cells (3), k h_bar,
              the refractive contrast sqrt(eps_in mu_in / eps_out) (1 for a PEC body);
      edge (m, n): (c_n - c_m)/h_bar (3), |c_n - c_m|/h_bar,
              N^A_mn / sqrt|N^A_mm N^A_nn|, N^Phi_mn / sqrt|N^Phi_mm N^Phi_nn|,
              h_bar N^K_mn / sqrt|N^A_mm N^A_nn|, k h_bar,
    with N the precorrected static near matrices (Eq. LAIMx).  Returns
    (x, e, rows, cols).
    """
    rwg, g = prob["rwg"], prob["grid"]
    h = np.asarray(g["h"], dtype=np.float64)
    hb = np.cbrt(h[0] * h[1] * h[2])
    k, contrast = _wavenumbers(freq, eps_out, eps_in, mu_in)
    N = prob["N"]
    c = rwg["center"]
    x = np.zeros((N, 8))
    x[:, 0] = rwg["length"] / hb
    x[:, 1] = rwg["area"][rwg["tp"]] / hb ** 2
    x[:, 2] = rwg["area"][rwg["tm"]] / hb ** 2
    x[:, 3:6] = (c - g["origin"]) / h - prob["anc"] - 0.5 * g["order"]
    x[:, 6] = k * hb
    x[:, 7] = contrast
    near = prob["near"]
    rows = near["rows"]
    cols = prob["cols"]
    dpos = rows == cols
    dA = np.zeros(N)
    dP = np.zeros(N)
    dA[rows[dpos]] = np.abs(near["NA"][dpos])
    dP[rows[dpos]] = np.abs(near["NP"][dpos])
    tiny = 1e-300
    sA = np.sqrt(np.maximum(dA[rows] * dA[cols], tiny))
    sP = np.sqrt(np.maximum(dP[rows] * dP[cols], tiny))
    e = np.zeros((len(rows), 8))
    d = (c[cols] - c[rows]) / hb
    e[:, 0:3] = d
    e[:, 3] = np.sqrt((d * d).sum(1))
    e[:, 4] = near["NA"] / sA
    e[:, 5] = near["NP"] / sP
    e[:, 6] = hb * near["NK"] / sA
    e[:, 7] = k * hb
    return x, e, rows, cols


def diag_inverse(prob, freq, eps_out=1.0, eps_in=None, mu_in=1.0):
    """D^{-1}: inverse of each basis' frequency-combined static self term (Sec. III-A-2).

    EFIE: [N] complex, 1 / (j w mu (L^A_s - L^Phi_s / k^2)).  Two-region form:
    [N, 2, 2], the inverse of [[sum_i j w mu_i <L_i>, 2 eta0 K_s], [-2 eta0 K_s,
    eta0^2 sum_i j w eps_i <L_i>]] on the self pair (unknowns [J; M/eta0])."""
    from .constants import MU0, EPS0, ETA0
    near = prob["near"]
    dpos = near["rows"] == prob["cols"]
    la, lp, kk = near["LsA_diag"], near["LsP_diag"], near["LsK_diag"]
    w = 2.0 * np.pi * freq
    regs = [(MU0, EPS0 * eps_out)]
    if eps_in is not None:
        regs.append((MU0 * mu_in, EPS0 * eps_in))
    order = near["rows"][dpos]
    if eps_in is None:
        mu, eps = regs[0]
        k2 = w * w * mu * eps
        d = 1j * w * mu * (la - lp / k2)
        out = np.empty(prob["N"], dtype=np.complex128)
        out[order] = 1.0 / d
        return out
    a = sum(1j * w * mu * (la - lp / (w * w * mu * eps)) for mu, eps in regs)
    dd = sum(ETA0 ** 2 * 1j * w * eps * (la - lp / (w * w * mu * eps)) for mu, eps in regs)
    b = 2.0 * ETA0 * kk
    c = -2.0 * ETA0 * kk
    blk = np.zeros((prob["N"], 2, 2), dtype=np.complex128)
    blk[order, 0, 0] = a
    blk[order, 0, 1] = b
    blk[order, 1, 0] = c
    blk[order, 1, 1] = dd
    return np.linalg.inv(blk)
