"""Oracle: Nystrom discretisation, dense solve and field evaluation.

TEST INFRASTRUCTURE ONLY.  Plain FP64 numpy.

Unknowns are the weighted densities phi~ = phi J (Section 3, Eq. (S:para))
at the nodes (t_i^n, th_l): panel i = 0..Np-1 (uniform panels of [0, L]),
Gauss-Legendre node n = 0..15, th_l = 2 pi l / Mth.  Flat index
(i*16 + n)*Mth + l.  On a torus-like surface (r(0, th) = r(L, th)) panel
indices are cyclic: panels 0 and Np-1 are adjacent (Section 3.1, Remark), and
the source nodes of a wrapped neighbour keep their unwrapped t (t < 0 or > L),
the surface being L-periodic in t.

Row of target (t_j^l, th_i), Section 3.1 Eq. (S123) and Section 3.4:
  far panels |i' - j| >= 2  (Eq. (S1) x Eq. (Sphi:sm)):
      A = (h/2) w_n (1/Mth) G~(x, y_{i',n,l'})
  near panels i' = j + delta, delta in {-1, 0, +1} (Section 3.4):
      A = sum_g (h/2) omega_g^{delta,l} L_n(s_g^{delta,l}) W_{l'}(pair g)
  with the 16-node GGQ rule (s_g, omega_g) of the table, L_n the Lagrange
  basis on the 16 Legendre nodes of panel i', and W_{l'} the Parseval
  weights of the pair's kernel: for the swapped part with modes K_m
      W_{l'} = (1/Mth) [ sum_{|m|<M} K_m e^{i m th_l'} + (K_M + K_{-M})/2 (-1)^{l'} ],
  plus, for the smooth part f (i sin(k rho)/rho, -i beta tau_0), f(th_l')/Mth.
Kernels G~: S -> e^{ik rho}/rho;  K -> tau_0 e^{ik rho}(ik rho - 1)/rho^3
(= alpha tau_1 - tau_3 - i beta tau_0, Section 4) with tau_0 = nu(y) . (y - x);
Kp (the adjoint K') -> the same with tau_0 = nu(x) . (x - y), the target's
normal (Eq. (adl)).

Operators acting on the weighted density (identity = diag(1/J)):
  "S"       S                     (Eq. (bie:S))
  "K"       K
  "K+I", "K-I"                    (Eq. (bie:Kie))
  "Kp", "Kp+I", "Kp-I"            (Eq. (bie:Kpie): + interior, - exterior Neumann)
  "CFIE"    I + K - i eta S       (exterior Dirichlet, combined field)
These are the paper's operators, which carry a factor 2 (Eqs. (sl), (adl)):
G~ omits 1/(4 pi) and the trapezoid weight 1/Mth omits 2 pi.
"""
import numpy as np

from . import geometry as geo
from . import kernel_modes as km

XG, WG = np.polynomial.legendre.leggauss(16)


def nodes(Np, L=np.pi):
    h = L / Np
    centers = (np.arange(Np) + 0.5) * h
    t = (centers[:, None] + (h / 2) * XG[None, :]).ravel()
    return t, h


def lagrange(x):
    """Lagrange basis on the 16 Gauss-Legendre nodes evaluated at x: (len(x), 16)."""
    x = np.atleast_1d(x)
    out = np.ones((len(x), 16))
    for n in range(16):
        for m in range(16):
            if m != n:
                out[:, n] *= (x - XG[m]) / (XG[n] - XG[m])
    return out


def parseval_weights_split(sing, smooth):
    """Weights of a kernel split into a swapped part (modes, symmetric Nyquist) and a smooth
    part (grid samples): for the smooth part the Fourier route is the trapezoid rule
    exactly (discrete Parseval, Section 3.2), so its weights are the samples / Mth."""
    return parseval_weights(sing) + smooth / smooth.shape[-1]


def parseval_weights(modes):
    """Physical theta weights W_l' from kernel modes K_m, m = -M..M (Section 3.4)."""
    M = (modes.shape[-1] - 1) // 2
    Mt = 2 * M
    th = 2 * np.pi * np.arange(Mt) / Mt
    m = np.arange(-M + 1, M)
    E = np.exp(1j * m[:, None] * th[None, :])
    W = modes[:, 1:2 * M] @ E
    W = W + 0.5 * (modes[:, :1] + modes[:, 2 * M:]) * ((-1.0) ** np.arange(Mt))[None, :]
    return W / Mt


def kernel_values(surface, x, t_s, th_s, k, kind, nu_x=None):
    """Point-to-surface kernel values G~ for target points x (..., 3)."""
    r, rt, rth, _, _, _ = geo.evaluate(surface, t_s, th_s)
    Y = r - x
    rho = np.sqrt(np.sum(Y * Y, -1))
    if kind == "S":
        return np.exp(1j * k * rho) / rho
    if kind == "Kp":
        tau0 = -np.sum(nu_x * Y, -1)
    else:
        nu, _ = geo.normal_and_jacobian(surface, t_s, th_s)
        tau0 = np.sum(nu * Y, -1)
    return tau0 * np.exp(1j * k * rho) * (1j * k * rho - 1) / rho ** 3


def near_pairs(Np, Mt, rows, ggq_x, L=np.pi, periodic=False):
    """Near pairs of the given target rows: list of (row, delta, g) plus t, th, t_s."""
    t_nodes, h = nodes(Np, L)
    out = []
    for r in rows:
        j, l, i = r // (16 * Mt), (r // Mt) % 16, r % Mt
        for di, delta in enumerate((-1, 0, 1)):
            ip = j + delta
            if not periodic and (ip < 0 or ip >= Np):
                continue
            for g in range(16):
                ts = (ip + 0.5) * h + (h / 2) * ggq_x[di, l, g]
                out.append((r, di, g, t_nodes[j * 16 + l], 2 * np.pi * i / Mt, ts))
    return out


def assemble_rows(surface, Np, Mt, k, ggq_x, ggq_w, rows, kinds=("S",), chunk=None, f_rule=False):
    """Dense rows of the S and/or K matrices: dict kind -> (len(rows), N).  Near pairs go through
    the per-pair pipeline in batches of `chunk` (default: about 200 MB of convolution table)."""
    if chunk is None:
        chunk = int(max(256, min(4096, 2e8 / (8 * (6 * Mt + 1) * (Mt + 1)))))
    L, periodic = geo.parameter_length(surface), geo.is_periodic(surface)
    t_nodes, h = nodes(Np, L)
    N = 16 * Np * Mt
    th = 2 * np.pi * np.arange(Mt) / Mt
    rows = np.asarray(rows)
    out = {kd: np.zeros((len(rows), N), complex) for kd in kinds}
    # far panels: Gauss-Legendre in t x trapezoid in theta
    TS = np.repeat(t_nodes, Mt)
    THS = np.tile(th, 16 * Np)
    src_panel = np.repeat(np.arange(Np), 16 * Mt)
    wq = np.repeat(np.tile(WG, Np), Mt) * (h / 2) / Mt
    tgt_panel = rows // (16 * Mt)
    X = geo.evaluate(surface, t_nodes[rows // Mt], th[rows % Mt])[0]
    NUX = geo.normal_and_jacobian(surface, t_nodes[rows // Mt], th[rows % Mt])[0] if "Kp" in kinds else None
    for c0 in range(0, len(rows), 64):
        sl = slice(c0, c0 + 64)
        dp = np.abs(src_panel[None, :] - tgt_panel[sl, None])
        far = (np.minimum(dp, Np - dp) if periodic else dp) >= 2
        for kd in kinds:
            with np.errstate(divide="ignore", invalid="ignore"):     # the self point is masked out
                vals = kernel_values(surface, X[sl, None, :], TS[None, :], THS[None, :], k, kd,
                                     NUX[sl, None, :] if kd == "Kp" else None)
            out[kd][sl] = np.where(far, wq[None, :] * vals, 0.0)
    # near panels: GGQ x Lagrange interpolation x Parseval weights
    coef = (h / 2) * ggq_w[..., None] * lagrange(ggq_x.ravel()).reshape(3, 16, 16, 16)
    pairs = near_pairs(Np, Mt, rows, ggq_x, L, periodic)
    row_pos = {r: p for p, r in enumerate(rows)}
    for c0 in range(0, len(pairs), chunk):
        block = pairs[c0:c0 + chunk]
        r = np.array([p[0] for p in block])
        di = np.array([p[1] for p in block])
        g = np.array([p[2] for p in block])
        t = np.array([p[3] for p in block])
        tht = np.array([p[4] for p in block])
        ts = np.array([p[5] for p in block])
        l = (r // Mt) % 16
        ip = (r // (16 * Mt) + di - 1) % Np
        pos = np.array([row_pos[v] for v in r])
        cols = ip[:, None, None] * 16 * Mt + np.arange(16)[None, :, None] * Mt + np.arange(Mt)[None, None, :]
        modes = km.method_modes(surface, t, tht, ts, Mt, k, kernels=tuple(kinds), f_rule=f_rule)
        for kd in kinds:
            W = parseval_weights_split(modes[kd + "_sing"], modes[kd + "_smooth"])
            vals = coef[di, l, g][:, :, None] * W[:, None, :]
            np.add.at(out[kd], (np.broadcast_to(pos[:, None, None], cols.shape), cols), vals)
    return out


def operator_rows(surface, Np, Mt, k, ggq_x, ggq_w, rows, op="S", eta=None, f_rule=False):
    """Rows of the operator matrix acting on the weighted density (f_rule: see method_modes)."""
    kinds = {"S": ("S",), "K": ("K",), "K+I": ("K",), "K-I": ("K",), "CFIE": ("S", "K"),
             "Kp": ("Kp",), "Kp+I": ("Kp",), "Kp-I": ("Kp",)}[op]
    blocks = assemble_rows(surface, Np, Mt, k, ggq_x, ggq_w, rows, kinds, f_rule=f_rule)
    if op == "S":
        return blocks["S"]
    A = blocks[kinds[0] if op.startswith("Kp") else "K"]
    if op in ("K", "Kp"):
        return A
    t_nodes, _ = nodes(Np, geo.parameter_length(surface))
    rows = np.asarray(rows)
    th = 2 * np.pi * np.arange(Mt) / Mt
    tr = t_nodes[rows // Mt]
    _, J = geo.normal_and_jacobian(surface, tr, th[rows % Mt])
    sign = {"K+I": 1.0, "K-I": -1.0, "Kp+I": 1.0, "Kp-I": -1.0, "CFIE": 1.0}[op]
    A[np.arange(len(rows)), rows] += sign / J
    if op == "CFIE":
        A = A - 1j * (k if eta is None else eta) * blocks["S"]
    return A


def boundary_nodes(surface, Np, Mt):
    t_nodes, h = nodes(Np, geo.parameter_length(surface))
    th = 2 * np.pi * np.arange(Mt) / Mt
    T = np.repeat(t_nodes, Mt)
    TH = np.tile(th, 16 * Np)
    r = geo.evaluate(surface, T, TH)[0]
    nu, J = geo.normal_and_jacobian(surface, T, TH)
    return r, nu, J, T, TH


def plane_wave_rhs(surface, Np, Mt, k, d):
    """Sound-soft data g = -e^{ik d.x} on the nodes."""
    r = boundary_nodes(surface, Np, Mt)[0]
    return -np.exp(1j * k * (r @ np.asarray(d, float)))


def point_source_rhs(surface, Np, Mt, k, src):
    """g = G(x; x_src) = e^{ik|x - x_src|}/(4 pi |x - x_src|) on the nodes."""
    r = boundary_nodes(surface, Np, Mt)[0]
    d = np.sqrt(np.sum((r - np.asarray(src)) ** 2, -1))
    return np.exp(1j * k * d) / (4 * np.pi * d)


def normal_derivative_rhs(surface, Np, Mt, k, src):
    """g = d/dnu(x) G(x; x_src) on the nodes (Neumann data of the point-source field)."""
    r, nu, _, _, _ = boundary_nodes(surface, Np, Mt)
    Y = r - np.asarray(src)
    d = np.sqrt(np.sum(Y * Y, -1))
    return np.sum(nu * Y, -1) * np.exp(1j * k * d) * (1j * k * d - 1) / (4 * np.pi * d ** 3)


def field(surface, Np, Mt, k, density, points, rep="S", eta=None):
    """u(x) at points off the surface (Section 3.4: GL in t x trapezoid in theta)."""
    t_nodes, h = nodes(Np, geo.parameter_length(surface))
    r, nu, J, T, TH = boundary_nodes(surface, Np, Mt)
    w = np.repeat(np.tile(WG, Np), Mt) * (h / 2) / Mt
    out = []
    for x in np.atleast_2d(points):
        Y = r - x
        rho = np.sqrt(np.sum(Y * Y, -1))
        gs = np.exp(1j * k * rho) / rho
        if rep == "S":
            kern = gs
        else:
            tau0 = np.sum(nu * Y, -1)
            kern = tau0 * np.exp(1j * k * rho) * (1j * k * rho - 1) / rho ** 3
            if rep == "CFIE":
                kern = kern - 1j * (k if eta is None else eta) * gs
        out.append(np.sum(w * kern * density))
    return np.array(out)


def far_field(surface, Np, Mt, k, density, dirs, rep="S", eta=None):
    """u_inf(d): u ~ e^{ik|x|}/|x| u_inf."""
    t_nodes, h = nodes(Np, geo.parameter_length(surface))
    r, nu, J, T, TH = boundary_nodes(surface, Np, Mt)
    w = np.repeat(np.tile(WG, Np), Mt) * (h / 2) / Mt
    out = []
    for d in np.atleast_2d(dirs):
        ph = np.exp(-1j * k * (r @ d))
        if rep == "S":
            kern = ph
        else:
            kern = -1j * k * (nu @ d) * ph
            if rep == "CFIE":
                kern = kern - 1j * (k if eta is None else eta) * ph
        out.append(np.sum(w * kern * density))
    return np.array(out)
