"""Oracle: theta-Fourier modes of the S and K kernels for near pairs.

TEST INFRASTRUCTURE ONLY.  Plain FP64 numpy, vectorised over a batch of
pairs.  A pair is (target point r(t, th), source curve t_s); its output is
the Fourier modes K_m, m = -M..M (M = Mth/2), of the kernel as a function
of the source angle th_s:

  S:  e^{ik rho}/rho                               (Section 3.2, Eq. (Sphi:appr2))
  K:  alpha tau_1 - tau_3 - i beta tau_0           (Section 4, Eq. (dis:K))
  Kp: the same with the roles of target and source exchanged in tau_j
      (Section 4, the K' integrand): tau_0 = nu(r) . (r - r_s), the normal of
      the target, again analytic in th_s and O(rho^2) at the target

``method_modes`` follows the paper's algorithm step by step:
  1. rho^2 on the Mth-point theta grid (Eq. (rho)); near samples use the
     cancellation-free line integral of the Section 4 Remark.
  2. a0 = real minimiser of rho^2, b0 = sqrt(2 rho^2(a0) / rho^2''(a0)),
     then complex Newton for the root theta_+ = a + i b (Section 3.3).
  3. F = (s_{a,b}/rho^2)^{1/2} (Lemma "singular1", Eq. (F-smooth)); modes.
  4. A_m(b) (Eq. (Am), special.a_modes); singular convolution
     <rho^{-1}>_l = sum_j <F>_j e^{-i(l-j)a} A_{|l-j|}  (Eq. (convolution)).
  5. S: <cos(k rho)> (x) <rho^{-1}> + i <sin(k rho)/rho>   (Eq. (Sphi:appr2)).
     K: <alpha> (x) (<tau_0> (x) <rho^{-1}>)  (Eqs. (dis:K), (tau1))
        - <tau_3> (Eq. (tau3-standard) for b >= 0.01, Eq. (tau3-modified)
        otherwise) - i <beta tau_0>.
Every smooth factor keeps all Mth of its grid modes (the paper's p and M_0
set to M), with the Nyquist mode split evenly between +M and -M.
Convolutions are written as direct sums.

``rho_inv_modes_banded`` and ``method_modes_banded`` follow the paper's other route to the modes
of 1/rho (Section 3.3, "An O(M) approach"): the difference equation Eq. (lin:diff) solved as the
banded system Eq. (Axb) with quadrature boundary values, then Eq. (Sphi:appr2) as in step 5.

``definition_modes`` is the plain definition <f>_m = (1/2pi) int f e^{-im th}
evaluated by the trapezoid rule on a grid refined until it converges
(brute force, no singularity swapping).
"""
import math
import numpy as np

from . import geometry as geo
from . import special as sp

STABLE_DELTA = 0.06     # |t - t_s| + |th - th_s| below which differences use the line integral
STABLE_DIST = 0.06      # ... or |r_s - r| below which they do (next to a pole, see _near_difference)
ROOT_TOL = 1e-14        # Newton stops when |dzeta| <= ROOT_TOL*b + 4e-16|zeta| (then one more step)
SERIES_X = 0.5          # alpha(rho), beta(rho) use their Taylor series when k rho < SERIES_X
SMALL_B = 0.1           # translated swapping for tau_3 when b < SMALL_B (the paper uses 0.01)
NEAR_PHI = 0.05         # |th_q - a| below which the translated remainder uses the stable sum
B_CAP = 4.0             # roots farther than this from the real axis are replaced by (a0, B_CAP)


# ----------------------------------------------------------------------------
# small helpers
# ----------------------------------------------------------------------------
def sym_modes(v, M):
    """Grid modes j = -M..M of samples v[..., 2M] (Nyquist split evenly)."""
    c = np.fft.fft(v, axis=-1) / (2 * M)
    out = np.zeros(v.shape[:-1] + (2 * M + 1,), complex)
    out[..., M:2 * M] = c[..., 0:M]
    out[..., 1:M] = c[..., M + 1:2 * M]
    out[..., 0] = c[..., M] / 2
    out[..., 2 * M] = c[..., M] / 2
    return out


def swap_convolution(f, a, A, lmax):
    """sum_j f_j e^{-i(l-j)a} A_{|l-j|} for l = -lmax..lmax  (Eq. (convolution)),
    written as e^{-ila} sum_j (f_j e^{ija}) A_{|l-j|} (the same sum, the phase split in two)."""
    M = (f.shape[-1] - 1) // 2
    j = np.arange(-M, M + 1)
    l = np.arange(-lmax, lmax + 1)
    d = l[:, None] - j[None, :]
    g = f * np.exp(1j * j[None, :] * a[:, None])
    return np.exp(-1j * l[None, :] * a[:, None]) * np.einsum("bj,blj->bl", g, A[:, np.abs(d)])


def linear_convolution(u, v, vmax, wmax):
    """w_m = sum_n u_n v_{m-n}, m = -wmax..wmax; u over -U..U, v over -vmax..vmax."""
    U = (u.shape[-1] - 1) // 2
    n = np.arange(-U, U + 1)
    m = np.arange(-wmax, wmax + 1)
    idx = m[:, None] - n[None, :]
    assert np.all(np.abs(idx) <= vmax)
    return np.einsum("bn,bmn->bm", u, v[:, idx + vmax])


def _series_coeffs():
    a = [(-1) ** (n + 1) * (1 - 2 * n) / math.factorial(2 * n) for n in range(1, 10)]
    b = [(-1) ** (n + 1) * (2 * n) / math.factorial(2 * n + 1) for n in range(1, 10)]
    return a, b


_ALPHA_C, _BETA_C = _series_coeffs()


def alpha_beta(rho, k):
    """alpha = (1 - cos k rho - k rho sin k rho)/rho^2, beta = (sin k rho - k rho cos k rho)/rho^3."""
    x = k * rho
    alpha = (1 - np.cos(x) - x * np.sin(x)) / rho ** 2
    beta = (np.sin(x) - x * np.cos(x)) / rho ** 3
    small = x < SERIES_X
    if np.any(small):
        xs2 = x[small] ** 2
        sa = sum(c * xs2 ** i for i, c in enumerate(_ALPHA_C))
        sb = sum(c * xs2 ** i for i, c in enumerate(_BETA_C))
        alpha[small] = k * k * sa
        beta[small] = k ** 3 * sb
    return alpha, beta


def _near_difference(surface, t_s, th_s, t, th):
    """r(t_s, th_s) - r(t, th) and the mask of samples that take the cancellation-free forms of the
    Section 4 Remark (line integrals for the difference and for tau_0): those within STABLE_DELTA in
    the parameters, or within STABLE_DIST in space.  The second test matters next to a pole, where J ~
    sin t vanishes: there a whole ring of source angles lies physically close to the target, and plain
    subtraction would give tau_0 ~ kappa rho^2 / 2 an absolute error ~eps |r|, i.e. a relative error
    ~2 eps |r| / (kappa rho^2) (1e-10 at rho = 1e-3).  For complex th_s the distance is the norm of the
    complex difference vector."""
    t_s, th_s, t, th = np.broadcast_arrays(np.asarray(t_s, float), np.asarray(th_s), np.asarray(t, float),
                                           np.asarray(th))
    Y = geo.evaluate(surface, t_s, th_s)[0] - geo.evaluate(surface, t, th)[0]
    par = np.abs(t_s - t) + np.abs(np.real(geo.wrap_angle(th_s - th))) <= STABLE_DELTA
    near = par | (np.sum(np.abs(Y) ** 2, -1) <= STABLE_DIST ** 2)
    if np.any(near):
        Y = Y.astype(np.result_type(Y, complex) if np.iscomplexobj(th_s) else Y.dtype)
        Y[near] = geo.difference(surface, t_s[near], th_s[near], t[near], th[near], True)
    return Y, near


# ----------------------------------------------------------------------------
# complex root of rho^2 (Section 3.3)
# ----------------------------------------------------------------------------
def locate_root(surface, t, th, t_s, thq, rho2):
    """a0, b0 and the Newton root (a, b) of rho^2(zeta) nearest to the real axis."""
    B, Mt = rho2.shape
    h = 2 * np.pi / Mt
    # grid minimiser; near-ties (within 1e-12) go to the sample nearest the target angle
    # (integer grid distance), then to the lower index, so rounding cannot pick a mirror root
    i_t = np.rint(th * Mt / (2 * np.pi)).astype(int) % Mt
    qq = np.arange(Mt)[None, :]
    dist = np.minimum(np.abs(qq - i_t[:, None]), Mt - np.abs(qq - i_t[:, None]))
    cand = rho2 <= rho2.min(axis=1, keepdims=True) * (1 + 1e-12)
    q = np.argmin(np.where(cand, dist * Mt + qq, 4 * Mt * Mt), axis=1)
    a0 = thq[q].copy()
    start = a0.copy()

    def deriv(z):
        Y, _ = _near_difference(surface, t_s, z, t, th)
        _, _, rth, _, _, rthth = geo.evaluate(surface, t_s, z)
        g0 = np.sum(Y * Y, -1)
        g1 = 2 * np.sum(Y * rth, -1)
        g2 = 2 * (np.sum(rth * rth, -1) + np.sum(Y * rthth, -1))
        return g0, g1, g2

    for _ in range(40):
        g0, g1, g2 = deriv(a0)
        step = np.where(g2 > 0, g1 / np.where(g2 > 0, g2, 1.0), 0.0)
        step = np.clip(step, -h, h)
        a0 = np.clip(a0 - step, start - h, start + h)
        if np.all(np.abs(step) <= 1e-15 * (1 + np.abs(a0))):
            break
    g0, g1, g2 = deriv(a0)
    b0 = np.sqrt(2 * g0 / np.where(g2 > 0, g2, 0.0))
    capped = ~(b0 <= B_CAP)
    zeta = a0 + 1j * np.where(capped, B_CAP, b0)
    done = capped.copy()
    extra = np.zeros(B, bool)
    for _ in range(60):
        g0, g1, _ = deriv(zeta)
        dz = g0 / g1
        upd = ~done
        zn = zeta - dz
        zn = np.where(zn.imag < 0, np.conj(zn), zn)
        over = upd & ~(zn.imag <= B_CAP)
        capped = capped | over
        zn = np.where(over, a0 + 1j * B_CAP, zn)
        zeta = np.where(upd, zn, zeta)
        small = np.abs(dz) <= ROOT_TOL * np.abs(zeta.imag) + 4e-16 * np.abs(zeta)
        done = done | over | (extra & upd)
        extra = extra | small
        if np.all(done):
            break
    return a0, b0, zeta.real, zeta.imag, done


# ----------------------------------------------------------------------------
# the method (singularity swapping)
# ----------------------------------------------------------------------------
def _pair_samples(surface, t, th, t_s, Mt):
    thq = 2 * np.pi * np.arange(Mt) / Mt
    T_s = np.broadcast_to(t_s[:, None], (len(t), Mt))
    TH_s = np.broadcast_to(thq[None, :], (len(t), Mt))
    T = np.broadcast_to(t[:, None], (len(t), Mt))
    TH = np.broadcast_to(th[:, None], (len(t), Mt))
    Y, near = _near_difference(surface, T_s, TH_s, T, TH)
    return thq, T_s, TH_s, T, TH, near, Y


def method_modes(surface, t, th, t_s, Mt, k, kernels=("S",), return_details=False, f_rule=False):
    """Kernel modes by singularity swapping; dict kernel -> (B, Mt+1) complex (m = -M..M).

    Also returns, per kernel, the swapped part "<kernel>_sing" (modes) and the
    smooth part "<kernel>_smooth" (its samples on the theta grid: i sin(k rho)/rho
    for S, -i beta tau_0 for K), whose Parseval weights are the trapezoid rule.

    By default F keeps the Mth modes of its grid samples (p = M, the reading the library's kernels
    follow).  With f_rule, p follows the paper's rule for the expansion of F (Eq. (F-expansion) with a
    criterion like Eq. (crt:M0)): F is sampled on grids of 2, 4, ... times Mth points until its modes
    at |j| >= p - 1 fall below 1e-14 of the largest, for surfaces where other complex roots of rho^2
    lie near the real axis and F needs more than Mth modes.
    """
    t = np.atleast_1d(np.asarray(t, float))
    th = np.atleast_1d(np.asarray(th, float))
    t_s = np.atleast_1d(np.asarray(t_s, float))
    M = Mt // 2
    thq, T_s, TH_s, T, TH, near, Y = _pair_samples(surface, t, th, t_s, Mt)
    rho2 = np.sum(Y * Y, -1)
    rho = np.sqrt(rho2)
    a0, b0, a, b, ok = locate_root(surface, t, th, t_s, thq, rho2)
    q = np.exp(-b)
    phi = thq[None, :] - a[:, None]
    s = (-np.expm1(-b))[:, None] ** 2 + 4 * q[:, None] * np.sin(phi / 2) ** 2   # Eq. (sab)
    F = np.sqrt(s / rho2)                                                     # Eq. (F-smooth)
    f = sym_modes(F, M)
    need_k = "K" in kernels or "Kp" in kernels
    L = (4 if need_k else 3) * M
    rmax = 3 * M if need_k else 2 * M
    if f_rule:
        p, qq = M, 1
        while qq < 16:
            tail = np.max(np.abs(np.concatenate([f[:, :2], f[:, -2:]], axis=1)), axis=1)
            if np.all(tail <= 1e-14 * np.max(np.abs(f), axis=1)):
                break
            qq *= 2
            n = qq * Mt
            thf = 2 * np.pi * np.arange(n) / n
            Tsf, THsf = np.broadcast_to(t_s[:, None], (len(t), n)), np.broadcast_to(thf[None, :], (len(t), n))
            Tf, THf = np.broadcast_to(t[:, None], (len(t), n)), np.broadcast_to(th[:, None], (len(t), n))
            Yf, _ = _near_difference(surface, Tsf, THsf, Tf, THf)
            sf = (-np.expm1(-b))[:, None] ** 2 + 4 * q[:, None] * np.sin((thf[None, :] - a[:, None]) / 2) ** 2
            p = qq * M
            f = sym_modes(np.sqrt(sf / np.sum(Yf * Yf, -1)), p)
        L = max(L, rmax + p + 1)
    A, D = sp.a_modes(b, L)
    out = {}
    R = swap_convolution(f, a, A, rmax)                                        # <rho^{-1}>_l
    if "S" in kernels:
        C = sym_modes(np.cos(k * rho), M)
        smooth = 1j * np.sin(k * rho) / rho
        out["S_sing"] = linear_convolution(C, R, rmax, M)
        out["S_smooth"] = smooth
        out["S"] = out["S_sing"] + sym_modes(smooth, M)
    if need_k:
        alpha, beta = alpha_beta(rho, k)
    for kd in ("K", "Kp"):
        if kd not in kernels:
            continue
        if kd == "K":   # source normal: nu(r_s) . (r_s - r)
            nu, _ = geo.normal_and_jacobian(surface, T_s, TH_s)
            tau0 = np.sum(nu * Y, -1)
            if np.any(near):
                tau0[near] = geo.tau0_stable(surface, T_s[near], TH_s[near], T[near], TH[near])
        else:           # target normal: nu(r) . (r - r_s)
            nu_x, _ = geo.normal_and_jacobian(surface, t, th)
            tau0 = -np.sum(nu_x[:, None, :] * Y, -1)
            if np.any(near):
                tau0[near] = geo.tau0_stable(surface, T[near], TH[near], T_s[near], TH_s[near])
        T0 = sym_modes(tau0, M)
        T1 = linear_convolution(T0, R, rmax, 2 * M)                            # Eq. (tau1)
        AT1 = linear_convolution(sym_modes(alpha, M), T1, 2 * M, M)
        T3 = tau3_modes(tau0 * F ** 3, a, b, A, D, M, (surface, t, th, t_s, f, kd == "Kp"))
        smooth = -1j * beta * tau0
        out[kd + "_sing"] = AT1 - T3
        out[kd + "_smooth"] = smooth
        out[kd] = out[kd + "_sing"] + sym_modes(smooth, M)
    if return_details:
        out["_a"], out["_b"], out["_a0"], out["_b0"], out["_ok"] = a, b, a0, b0, ok
        out["_R"], out["_rmax"] = R, rmax
    return out


def tau3_modes(H3, a, b, A, D, M, pair):
    """<tau_3>_n, n = -M..M, from H3 = tau_0 F^3 (Eqs. (tau3-standard), (tau3-modified))."""
    Bn = sp.b_modes(b, A[:, :2 * M + 2], D[:, :2 * M + 2])                  # B_m(0,b), m = 0..2M+1
    h3 = sym_modes(H3, M)
    out = swap_convolution(h3, a, Bn, M)                                       # standard form
    small = b < SMALL_B
    if np.any(small):
        i = np.nonzero(small)[0]
        surface, t, th, t_s, f = pair[:5]
        target_normal = len(pair) > 5 and pair[5]
        Ha, H1a = h3_at_root(surface, t[i], th[i], t_s[i], a[i], b[i], f[i], target_normal)
        out[i] = _tau3_translated(H3[i], h3[i], a[i], b[i], A[i], Bn[i], M, Ha, H1a)
    return out


def h3_at_root(surface, t, th, t_s, a, b, f=None, target_normal=False):
    """H3(a) = tau_0(a) F(a)^3 and H3'(a), evaluated at th_s = a.

    tau_0(a), tau_0'(a) = nu'(a) . (r_s(a) - r) and F(a) = (1 - e^{-b}) / rho(a)
    (s_{a,b}(a) = (1 - e^{-b})^2) come directly from the geometry: they are
    small (O(b^2), O(b), O(1)) and only a direct evaluation is relatively
    accurate.  With target_normal (the K' integrand) tau_0 = nu(r) . (r - r_s(a))
    and tau_0'(a) = -nu(r) . r_th(t_s, a).  F'(a) comes from the trigonometric interpolant of F (modes f):
    F is smooth, while the direct form -F (rho^2)'(a) / (2 rho^2(a)) divides an
    O(b^2) dot product of O(b) vectors by rho^2 and loses digits like eps/b.
    """
    Y, near = _near_difference(surface, t_s, a, t, th)
    _, rt, rth, _, rtth, rthth = geo.evaluate(surface, t_s, a)
    if target_normal:
        nu_x, _ = geo.normal_and_jacobian(surface, t, th)
        tau0 = -np.sum(nu_x * Y, -1)
        if np.any(near):
            tau0[near] = geo.tau0_stable(surface, t[near], th[near], t_s[near], a[near])
        dtau0 = -np.sum(nu_x * rth, -1)
    else:
        n = np.cross(rt, rth)
        J = np.sqrt(np.sum(n * n, -1))
        nu = n / J[:, None]
        dn = np.cross(rtth, rth) + np.cross(rt, rthth)
        dnu = (dn - nu * np.sum(nu * dn, -1)[:, None]) / J[:, None]
        tau0 = np.sum(nu * Y, -1)
        if np.any(near):
            tau0[near] = geo.tau0_stable(surface, t_s[near], a[near], t[near], th[near])
        dtau0 = np.sum(dnu * Y, -1)
    rho2 = np.sum(Y * Y, -1)
    F = -np.expm1(-b) / np.sqrt(rho2)
    if f is None:
        dF = -F * np.sum(Y * rth, -1) / rho2
    else:
        M = (f.shape[-1] - 1) // 2
        j = np.arange(-M, M + 1)
        dF = np.real(np.sum(f * (1j * j)[None, :] * np.exp(1j * j[None, :] * a[:, None]), -1))
    return tau0 * F ** 3, dtau0 * F ** 3 + 3 * tau0 * F ** 2 * dF


def _tau3_translated(H3, h3, a, b, A, Bn, M, H_a, H1_a):
    """Translated singularity swapping for small b (Section 4, Eq. (tau3-modified))."""
    Mt = 2 * M
    kk = np.arange(-M, M + 1)
    e = np.exp(1j * kk[None, :] * a[:, None])
    thq = 2 * np.pi * np.arange(Mt) / Mt
    phi = geo.wrap_angle(thq[None, :] - a[:, None])
    close = np.abs(phi) < NEAR_PHI
    den = np.where(close, 1.0, np.sin(phi / 2) ** 2)
    Rs = (H3 - H_a[:, None] - H1_a[:, None] * np.sin(phi)) / den
    for bi, qi in zip(*np.nonzero(close)):
        p = phi[bi, qi]
        s2 = np.sin(p / 2) ** 2
        if s2 == 0.0:            # the limit 2 H3''(a)
            Rs[bi, qi] = np.real(np.sum(-2 * kk * kk * h3[bi] * e[bi]))
            continue
        acc = 0.0
        for kv, hv in zip(kk, h3[bi] * e[bi]):
            kabs = abs(kv)
            re = -2 * np.sin(kabs * p / 2) ** 2 / s2 if kabs else 0.0
            # sin(k p) - k sin(p) = -2 sin(p) sum_{j<k} sin^2((k-1-2j) p/2)
            ssum = sum(np.sin((kabs - 1 - 2 * j) * p / 2) ** 2 for j in range(kabs))
            im = np.sign(kv) * (-2 * np.sin(p) * ssum) / s2
            acc = acc + hv * (re + 1j * im)
        Rs[bi, qi] = np.real(acc)
    d = sym_modes(Rs, M)
    q = np.exp(-b)
    om2 = np.expm1(-b) ** 2
    Lb = Bn.shape[1] - 1
    m = np.arange(-Lb, Lb + 1)
    Bfull = Bn[:, np.abs(m)] * np.exp(-1j * m[None, :] * a[:, None])        # B_m(a, b)
    Btil = (A[:, :Lb + 1] - om2[:, None] * Bn) / (4 * q[:, None])            # B~_m(0, b), m = 0..Lb
    n = np.arange(-M, M + 1)
    c = Lb
    out = H_a[:, None] * Bfull[:, n + c]
    # H3'(a)/(2i) [e^{-ia} B_{n-1}(a,b) - e^{ia} B_{n+1}(a,b)] = H3'(a)/(2i) e^{-ina} (B_{|n-1|} - B_{|n+1|}),
    # and B_{n-1} - B_{n+1} = <2i sin(th) s^{-3/2}>_n = 2 n e^b A_{|n|} by the identity
    # d/dth s^{-1/2} = -e^{-b} sin(th) s^{-3/2} (proof of Prop. "lem:Bm"); the difference of two
    # O(1/b^2) numbers would lose ~log10(1/b^2) digits for small b.
    phase = np.exp(-1j * n[None, :] * a[:, None])
    out = out + (H1_a / 2j)[:, None] * phase * (2 * n[None, :] * np.exp(b)[:, None] * A[:, np.abs(n)])
    out = out + swap_convolution(d, a, Btil, M)
    return out


# ----------------------------------------------------------------------------
# the O(M) route to <rho^{-1}>_l (Section 3.3, the "O(M) approach")
# ----------------------------------------------------------------------------
def rho_inv_modes_banded(surface, t, th, t_s, lmax, eps0=1e-14):
    """<rho^{-1}>_l, l = 0..lmax, of one pair (t != t_s) from the difference equation Eq. (lin:diff).

    Steps as the paper orders them:
      1. <rho^2>_n by the trapezoid rule (rho^2 is analytic and periodic in th_s), and m0 by
         Eq. (crt:M0), read as a bound on the whole tail: the smallest m0 with |<rho^2>_n| <=
         eps0 max_k |<rho^2>_k| for every |n| > m0 (surfaces whose rho^2 skips some modes, like
         the bumpy star, have isolated zero modes that the literal test at +-m0 alone would stop at);
      2. the 2 m0 boundary values <rho^{-1}>_0..m0-1 and <rho^{-1}>_{lmax-m0+1}..lmax
         (Eq. (offline:terms)) by quadrature (here the refined trapezoid of the definition);
      3. a_j(i) = (m0 + 2i + j) <rho^2>_{m0-j} (Eq. (def:a_l)), i = 0..M1 = lmax - 2 m0, and the
         banded system A x = b (Eq. (Axb)) for x = <rho^{-1}>_{m0}..<rho^{-1}>_{lmax-m0}, the
         boundary values moved to b; A is Hermitian with band 2 m0 + 1 (Lemma after Eq. (root:x)).
    Returns (modes [lmax+1], m0).
    """
    # 1. modes of rho^2 (a trigonometric polynomial of low degree on the surfaces used here; the grid
    #    is refined until the modes stop changing)
    n = 64
    prev = None
    while True:
        thq = 2 * np.pi * np.arange(n) / n
        Y, near = _near_difference(surface, np.full(n, t_s), thq, np.full(n, t), np.full(n, th))
        c = np.fft.fft(np.sum(Y * Y, -1)) / n
        if prev is not None and np.max(np.abs(c[:32] - prev[:32])) <= 1e-16 * np.max(np.abs(c)):
            break
        prev = np.concatenate([c[: n // 2], np.zeros(n // 2)])
        n *= 2
    rho2 = lambda k: c[k % n]
    big = np.max(np.abs(c))
    m0 = n // 4
    while m0 > 1 and max(abs(rho2(m0)), abs(rho2(-m0))) <= eps0 * big:
        m0 -= 1
    # 2. boundary values by quadrature of the definition
    M = lmax
    R, _ = definition_rho_inv(surface, t, th, t_s, M)          # <rho^{-1}>_l, l = -M..M
    out = np.zeros(lmax + 1, complex)
    lo = list(range(0, m0))
    hi = list(range(lmax - m0 + 1, lmax + 1))
    for l in lo + hi:
        out[l] = R[M + l]
    # 3. the banded system: equation i couples <rho^{-1}>_{i..i+2 m0}
    M1 = lmax - 2 * m0
    A = np.zeros((M1 + 1, M1 + 1), complex)
    b = np.zeros(M1 + 1, complex)
    for i in range(M1 + 1):
        for j in range(2 * m0 + 1):
            a = (m0 + 2 * i + j) * rho2(m0 - j)
            col = i + j - m0                                      # unknown x_col = <rho^{-1}>_{i+j}
            if 0 <= col <= M1:
                A[i, col] += a
            else:
                b[i] -= a * out[i + j]
    out[m0:lmax - m0 + 1] = np.linalg.solve(A, b)
    return out, m0


def method_modes_banded(surface, t, th, t_s, Mt, k, eps0=1e-14):
    """Single-layer modes K_m, m = -M..M, through the O(M) route: Eq. (Sphi:appr2) with M_0 = M, the
    modes of 1/rho for |l| <= 2M from rho_inv_modes_banded (Eq. (lin:diff)), the grid modes of cos(k rho)
    and of the smooth part i sin(k rho)/rho as in method_modes.  Returns (B, Mt+1) complex."""
    t = np.atleast_1d(np.asarray(t, float))
    th = np.atleast_1d(np.asarray(th, float))
    t_s = np.atleast_1d(np.asarray(t_s, float))
    M = Mt // 2
    thq = 2 * np.pi * np.arange(Mt) / Mt
    out = np.zeros((len(t), Mt + 1), complex)
    for i in range(len(t)):
        Y, _ = _near_difference(surface, np.full(Mt, t_s[i]), thq, np.full(Mt, t[i]), np.full(Mt, th[i]))
        rho = np.sqrt(np.sum(Y * Y, -1))
        Rp, _ = rho_inv_modes_banded(surface, t[i], th[i], t_s[i], 2 * M, eps0)
        R = np.concatenate([np.conj(Rp[:0:-1]), Rp])[None, :]                # l = -2M..2M
        C = sym_modes(np.cos(k * rho), M)[None, :]
        out[i] = linear_convolution(C, R, 2 * M, M)[0] + sym_modes(1j * np.sin(k * rho) / rho, M)
    return out


def definition_rho_inv(surface, t, th, t_s, M, tol=1e-15, n_max=2 ** 22):
    """<rho^{-1}>_m, m = -M..M, by the trapezoid rule refined until converged (plain definition)."""
    n = max(8 * M, 64)
    prev = None
    while True:
        thq = 2 * np.pi * np.arange(n) / n
        Y, near = _near_difference(surface, np.full(n, t_s), thq, np.full(n, t), np.full(n, th))
        c = np.fft.fft(1.0 / np.sqrt(np.sum(Y * Y, -1))) / n
        m = np.arange(-M, M + 1)
        cur = c[m % n]
        if (prev is not None and np.max(np.abs(cur - prev)) <= tol * np.max(np.abs(cur))) or n >= n_max:
            return cur, n
        prev = cur
        n *= 2


# ----------------------------------------------------------------------------
# the plain definition (brute force)
# ----------------------------------------------------------------------------
def definition_modes(surface, t, th, t_s, M, k, kernel="S", n_start=None, tol=1e-15, n_max=2 ** 22):
    """<f>_m, m = -M..M, by the trapezoid rule refined until converged."""
    n = n_start or max(8 * M, 64)
    prev = None
    while True:
        thq = 2 * np.pi * np.arange(n) / n
        Y, near = _near_difference(surface, np.full(n, t_s), thq, np.full(n, t), np.full(n, th))
        rho = np.sqrt(np.sum(Y * Y, -1))
        if kernel == "S":
            f = np.exp(1j * k * rho) / rho
        elif kernel == "K":
            nu, _ = geo.normal_and_jacobian(surface, np.full(n, t_s), thq)
            tau0 = np.sum(nu * Y, -1)
            if np.any(near):
                tau0[near] = geo.tau0_stable(surface, np.full(near.sum(), t_s), thq[near],
                                             np.full(near.sum(), t), np.full(near.sum(), th))
            f = tau0 * np.exp(1j * k * rho) * (1j * k * rho - 1) / rho ** 3
        else:   # Kp: the target's normal
            nu_x, _ = geo.normal_and_jacobian(surface, t, th)
            tau0 = -(Y @ nu_x)
            if np.any(near):
                tau0[near] = geo.tau0_stable(surface, np.full(near.sum(), t), np.full(near.sum(), th),
                                             np.full(near.sum(), t_s), thq[near])
            f = tau0 * np.exp(1j * k * rho) * (1j * k * rho - 1) / rho ** 3
        c = np.fft.fft(f) / n
        m = np.arange(-M, M + 1)
        cur = c[m % n]
        if prev is not None and np.max(np.abs(cur - prev)) <= tol * np.max(np.abs(cur)):
            return cur, n
        if n >= n_max:
            return cur, n
        prev = cur
        n *= 2
