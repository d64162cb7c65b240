"""FP64 reference of the learned near-field preconditioner network (test infrastructure).

Only tests, the smoke check and the benchmark's CPU baseline may import this module.

Not in the paper: the paper's preconditioner is the diagonal of L_s, and it
notes that off-diagonal entries may augment it (Sec. III-A-2).  The learned
form used by the library is

    M = D^{-1} (I + C),   C supported on the near-region graph (and its diagonal),

with D the per-basis frequency-combined static self block.  Reversing the
orientation of RWG function n multiplies row and column n of A by -1, and the
ideal C transforms the same way (C_mn -> s_m s_n C_mn).  The network is built
to respect that: its node states see only orientation-invariant inputs, and an
edge entry is a learned combination of signed bases b_c(m, n) that carry the
transformation,

    C_mn[k] = sum_c w_mn[k, c] b_c(m, n),   w_mn = E u_mn + f,
    u_mn    = relu(Ua h_m + Ub h_n + Uc e_mn + u),
    C_mm[k] = G h_m + g,

where the node states come from message passing over the near graph:

    h0   = relu(A0 x_m + a0)
    q_mn = relu(B_l h_n + C_l e_mn + c_l)                 (edges n -> m, n != m)
    h_l  = relu(D_l h_m + (1/deg_m) sum_n q_mn + d_l),     l = 1..L.

Bases (8): the normalised static near entries eta^A, eta^Phi, eta^K
(Eq. LAIMx's N, scaled by the self terms) and their two-hop products AA, PP,
AP, PA, KK on the near pattern.  K = 2 (one complex entry, EFIE) or 8 (a 2x2
complex block of the two-region form, row-major (E,J), (E,M), (H,J), (H,M),
real parts then imaginary parts).  Training minimises the probe loss

    L = (1/P) sum_p |M y_p - z_p|^2 / |z_p|^2,   y_p = A z_p,

which is quadratic in C, so A is only needed through the fixed pairs (z, y).

This module computes the features, the forward pass, the loss and all
parameter gradients in float64 (explicit backpropagation); tests pin the
gradients with central finite differences and compare the CUDA kernels with
it.
"""

import numpy as np

NIN = 8      # node features
NED = 16     # edge features (orientation invariant)
NB = 8       # signed bases
BASES = ("A", "P", "K", "AA", "PP", "AP", "PA", "KK")


def param_order(layers=4):
    return ["A0", "a0"] + [f"{n}{l}" for l in range(1, layers + 1) for n in ("B", "C", "c", "D", "d")] + \
        ["Ua", "Ub", "Uc", "u", "E", "f", "G", "g"]


PARAM_ORDER = param_order(4)


def param_shapes(width=64, layers=4, K=2):
    s = {"A0": (width, NIN), "a0": (width,)}
    for l in range(1, layers + 1):
        s[f"B{l}"] = (width, width)
        s[f"C{l}"] = (width, NED)
        s[f"c{l}"] = (width,)
        s[f"D{l}"] = (width, width)
        s[f"d{l}"] = (width,)
    s.update({"Ua": (width, width), "Ub": (width, width), "Uc": (width, NED), "u": (width,),
              "E": (K * NB, width), "f": (K * NB,), "G": (K, width), "g": (K,)})
    return s


def relu(v):
    return np.maximum(v, 0.0)


# ------------------------------------------------------------------ forward

def forward(params, x, e, basis, rows, cols, layers=4):
    """x [N, 8], e [nnz, 16], basis [nnz, 8] per stored near pair (diagonal included, skipped).

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
        h.append(relu(hp @ params[f"D{l}"].T + s + params[f"d{l}"]))
        cache["w"].append(w)
    hL = h[-1]
    z = (hL @ params["Ua"].T)[rows] + (hL @ params["Ub"].T)[cols] + e @ params["Uc"].T + params["u"]
    U = relu(z)
    K = params["G"].shape[0]
    W = (U @ params["E"].T + params["f"]).reshape(-1, K, NB)
    o = np.einsum("ekc,ec->ek", W, basis) * off[:, None]
    g = hL @ params["G"].T + params["g"]
    cache.update(h=h, U=U)
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


# ------------------------------------------------------------------ loss and gradients

def loss_and_grads(params, x, e, basis, rows, cols, dinv, Y, Zp, K, layers=4):
    """Probe loss and gradients of every parameter (dict), float64."""
    o, g, cache = forward(params, x, e, basis, rows, cols, layers)
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
    hL, U = h[-1], cache["U"]
    # edge head
    dW = (G_e[:, :, None] * basis[:, None, :]).reshape(len(rows), K * NB)
    grads["E"] = dW.T @ U
    grads["f"] = dW.sum(0)
    dz = (dW @ params["E"]) * (U > 0)
    grads["Uc"] = dz.T @ e
    grads["u"] = dz.sum(0)
    dza = np.zeros_like(hL)
    dzb = np.zeros_like(hL)
    np.add.at(dza, rows, dz)
    np.add.at(dzb, cols, dz)
    grads["Ua"] = dza.T @ hL
    grads["Ub"] = dzb.T @ hL
    # diagonal head
    grads["G"] = G_n.T @ hL
    grads["g"] = G_n.sum(0)
    dh = dza @ params["Ua"] + dzb @ params["Ub"] + G_n @ params["G"]
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


def init_params(seed, width=64, layers=4, K=2):
    """He-style initialisation; E, f, G, g start at zero so C = 0 (the diagonal preconditioner)."""
    rng = np.random.default_rng(seed)
    out = {}
    for k, shp in param_shapes(width, layers, K).items():
        if len(shp) == 2 and k not in ("E", "G"):
            out[k] = rng.standard_normal(shp) * np.sqrt(2.0 / shp[1])
        else:
            out[k] = np.zeros(shp)
    return out


# ------------------------------------------------------------------ inputs of the network

def _wavenumber(freq, eps_out, eps_in, mu_in):
    from .constants import C0
    k_out = 2.0 * np.pi * freq * np.sqrt(eps_out) / C0
    contrast = 1.0 if eps_in is None else np.sqrt(eps_in * mu_in / eps_out)
    return k_out, contrast


def features(prob, freq, eps_out=1.0, eps_in=None, mu_in=1.0):
    """Node features x [N, 8], edge features e [nnz, 16] and signed bases [nnz, 8] (caller order).

    With h_bar the geometric mean of the grid spacings and k the exterior
    wavenumber, every quantity is dimensionless:

      node m: l_m/h_bar, A+_m/h_bar^2, A-_m/h_bar^2, the offset of the basis
              centre from the stencil's central node in cells (3), k h_bar,
              the refractive contrast sqrt(eps_in mu_in / eps_out) (1 for a PEC body);
      bases (m, n): eta^A = N^A_mn / sqrt|N^A_mm N^A_nn|,
              eta^Phi = N^Phi_mn / sqrt|N^Phi_mm N^Phi_nn|,
              eta^K = h_bar N^K_mn / sqrt|N^A_mm N^A_nn|,
              and the two-hop products (XY)_mn = sum_j X_mj Y_jn / sqrt(deg_m deg_n)
              over the near pattern (diagonal included) for XY = AA, PP, AP, PA, KK,
              deg the off-diagonal near count (at least 1);
      edge (m, n): (c_n - c_m)/h_bar (3), |c_n - c_m|/h_bar, |eta^A|, |eta^Phi|,
              eta^A eta^Phi, |eta^K|, |AA|, |PP|, |AP|, |PA|, |KK|, eta^A AA,
              eta^Phi PP, k h_bar,
    with N the precorrected static near matrices (Eq. LAIMx).  Returns
    (x, e, basis, rows, cols).
    """
    import scipy.sparse as sp
    rwg, g = prob["rwg"], prob["grid"]
    h = np.asarray(g["h"], dtype=np.float64)
    hb = np.cbrt(h[0] * h[1] * h[2])
    k, contrast = _wavenumber(freq, eps_out, eps_in, mu_in)
    N = prob["N"]
    c = rwg["center"]
    x = np.zeros((N, NIN))
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
    eta = {"A": near["NA"] / sA, "P": near["NP"] / sP, "K": hb * near["NK"] / sA}
    deg = np.maximum(np.bincount(rows[~dpos], minlength=N), 1).astype(np.float64)
    nrm = 1.0 / np.sqrt(deg[rows] * deg[cols])
    mats = {a: sp.csr_matrix((eta[a], (rows, cols)), shape=(N, N)) for a in eta}
    basis = np.zeros((len(rows), NB))
    for i, name in enumerate(BASES):
        if len(name) == 1:
            basis[:, i] = eta[name]
        else:
            prod = (mats[name[0]] @ mats[name[1]]).tocsr()
            basis[:, i] = np.asarray(prod[rows, cols]).ravel() * nrm
    d = (c[cols] - c[rows]) / hb
    e = np.zeros((len(rows), NED))
    e[:, 0:3] = d
    e[:, 3] = np.sqrt((d * d).sum(1))
    e[:, 4] = np.abs(basis[:, 0])
    e[:, 5] = np.abs(basis[:, 1])
    e[:, 6] = basis[:, 0] * basis[:, 1]
    e[:, 7] = np.abs(basis[:, 2])
    e[:, 8:13] = np.abs(basis[:, 3:8])
    e[:, 13] = basis[:, 0] * basis[:, 3]
    e[:, 14] = basis[:, 1] * basis[:, 4]
    e[:, 15] = k * hb
    return x, e, basis, rows, cols


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
