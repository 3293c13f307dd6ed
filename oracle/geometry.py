"""Oracle: analytic surfaces r(t, theta) and their derivatives (Section 2, Eq. (para)).

TEST INFRASTRUCTURE ONLY.  Plain FP64 numpy; slow and direct.

A surface is described by a plain dict (produced by the seeded input
generators in ``workloads``):

  {"kind": "ellipsoid", "axes": (a, b, c)}
      r = (a sin t cos th, b sin t sin th, c cos t),  t in [0, pi]
  {"kind": "star", "terms": [[c, p, q, m, s], ...]}
      r = h(t, th) (sin t cos th, sin t sin th, cos t),
      h = 1 + sum_i c_i sin^p_i(t) cos^q_i(t) T_i(m_i th),
      T = cos if s_i == 0 else sin,  t in [0, pi]
  {"kind": "bean"}
      the bean of Section 5, Example 2 (given implicitly there): at height
      z = cos t the surface is the ellipse x^2/A + (y + 0.3 cos(pi z))^2/B = 1 - z^2,
      A = 0.64 (1 - 0.1 cos(pi z)), B = 0.64 (1 - 0.4 cos(pi z)), so
      r = (sqrt(A) sin t cos th, -0.3 cos(pi z) + sqrt(B) sin t sin th, z),  t in [0, pi]
  {"kind": "fourier_torus", "R": R, "terms": [[c, m, n], ...]}
      r = (w cos t, w sin t, zeta),  w = R + sum c cos(m th + n t),
      zeta = sum c sin(m th + n t),  t in [0, 2 pi] periodic (the twisted torus
      of Section 5, Example 4, has R = 4.5 and the six terms printed there)
  {"kind": "torus", "a": a, "b": b, "c": c, "R": R, "eps": eps, "m": m}
      r = (a w cos t, b w sin t, c sin th),  w = R + cos th + eps cos(m t),
      t in [0, 2 pi] with r(0, th) = r(2 pi, th): a torus-like surface (the
      wiggly torus of Section 5, Example 3, has a, b, c, R, eps, m =
      1.2, 1, 1.7, 2, 0.25, 5)

All satisfy assumptions (i)-(iii) of Section 2 at every quadrature node (J
vanishes only at the poles t = 0, pi of the first two, which are never nodes;
it does not vanish on the torus).

Every function accepts real t and real or complex theta (complex theta is
the analytic continuation used to locate the complex root of rho^2,
Section 3.3).
"""
import numpy as np


def parameter_length(surface):
    """Length L of the t-interval [0, L] (Section 2)."""
    return 2 * np.pi if surface["kind"] in ("torus", "fourier_torus") else np.pi


def is_periodic(surface):
    """Torus-like surface (r(0, th) = r(L, th)): the first and last panels are adjacent (Section 3.1)."""
    return surface["kind"] in ("torus", "fourier_torus")


def _sc_power(st, ct, p, q):
    """sin^p cos^q with the convention that a zero exponent gives 1."""
    out = np.ones_like(st)
    if p:
        out = out * st ** p
    if q:
        out = out * ct ** q
    return out


def _star_h(terms, t, th):
    """h and its first and second partial derivatives."""
    st, ct = np.sin(t), np.cos(t)
    h = np.ones(np.broadcast(t, th).shape, dtype=np.result_type(t, th, float))
    ht = np.zeros_like(h); hth = np.zeros_like(h)
    htt = np.zeros_like(h); htth = np.zeros_like(h); hthth = np.zeros_like(h)
    for c, p, q, m, s in terms:
        p, q, m = int(p), int(q), int(m)
        g = _sc_power(st, ct, p, q)
        # d/dt sin^p cos^q = p sin^(p-1) cos^(q+1) - q sin^(p+1) cos^(q-1)
        gt = 0.0
        if p:
            gt = gt + p * _sc_power(st, ct, p - 1, q + 1)
        if q:
            gt = gt - q * _sc_power(st, ct, p + 1, q - 1)
        gtt = 0.0
        if p:
            if p - 1:
                gtt = gtt + p * (p - 1) * _sc_power(st, ct, p - 2, q + 2)
            gtt = gtt - p * (q + 1) * _sc_power(st, ct, p, q)
        if q:
            gtt = gtt - q * (p + 1) * _sc_power(st, ct, p, q)
            if q - 1:
                gtt = gtt + q * (q - 1) * _sc_power(st, ct, p + 2, q - 2)
        if int(s) == 0:
            T, Tth, Tthth = np.cos(m * th), -m * np.sin(m * th), -m * m * np.cos(m * th)
        else:
            T, Tth, Tthth = np.sin(m * th), m * np.cos(m * th), -m * m * np.sin(m * th)
        h = h + c * g * T
        ht = ht + c * gt * T
        hth = hth + c * g * Tth
        htt = htt + c * gtt * T
        htth = htth + c * gt * Tth
        hthth = hthth + c * g * Tthth
    return h, ht, hth, htt, htth, hthth


def evaluate(surface, t, th):
    """Return r, r_t, r_th, r_tt, r_tth, r_thth as arrays of shape (..., 3)."""
    t = np.asarray(t, float)
    th = np.asarray(th)
    st, ct = np.sin(t), np.cos(t)
    sp, cp = np.sin(th), np.cos(th)
    st, ct, sp, cp = np.broadcast_arrays(st, ct, sp, cp)
    z = np.zeros(st.shape, dtype=np.result_type(st, sp))
    if surface["kind"] == "ellipsoid":
        a, b, c = surface["axes"]
        r = np.stack([a * st * cp, b * st * sp, c * ct + z], -1)
        rt = np.stack([a * ct * cp, b * ct * sp, -c * st + z], -1)
        rth = np.stack([-a * st * sp, b * st * cp, z], -1)
        rtt = np.stack([-a * st * cp, -b * st * sp, -c * ct + z], -1)
        rtth = np.stack([-a * ct * sp, b * ct * cp, z], -1)
        rthth = np.stack([-a * st * cp, -b * st * sp, z], -1)
        return r, rt, rth, rtt, rtth, rthth
    if surface["kind"] == "star":
        h, ht, hth, htt, htth, hthth = _star_h(surface["terms"], t, th)
        e = np.stack([st * cp, st * sp, ct + z], -1)
        et = np.stack([ct * cp, ct * sp, -st + z], -1)
        eth = np.stack([-st * sp, st * cp, z], -1)
        ett = -e
        etth = np.stack([-ct * sp, ct * cp, z], -1)
        ethth = np.stack([-st * cp, -st * sp, z], -1)
        H = lambda v: np.asarray(v)[..., None]
        r = H(h) * e
        rt = H(ht) * e + H(h) * et
        rth = H(hth) * e + H(h) * eth
        rtt = H(htt) * e + 2 * H(ht) * et + H(h) * ett
        rtth = H(htth) * e + H(ht) * eth + H(hth) * et + H(h) * etth
        rthth = H(hthth) * e + 2 * H(hth) * eth + H(h) * ethth
        return r, rt, rth, rtt, rtth, rthth
    if surface["kind"] == "bean":
        # u = cos(pi z), z = cos t; p(t) = sqrt(A) sin t, q(t) = sqrt(B) sin t, y0(t) = -0.3 u
        u = np.cos(np.pi * ct)
        du = np.pi * st * np.sin(np.pi * ct)                            # d/dt cos(pi cos t)
        ddu = np.pi * ct * np.sin(np.pi * ct) - (np.pi * st) ** 2 * u
        def ellipse_factor(c0):
            # f = 0.8 sqrt(1 - c0 u) sin t and its first two t-derivatives
            g = 1 - c0 * u
            sg = np.sqrt(g)
            dg, ddg = -c0 * du, -c0 * ddu
            dsg = dg / (2 * sg)
            ddsg = ddg / (2 * sg) - dg * dg / (4 * g * sg)
            return 0.8 * sg * st, 0.8 * (dsg * st + sg * ct), 0.8 * (ddsg * st + 2 * dsg * ct - sg * st)
        pf, pt, ptt = ellipse_factor(0.1)
        qf, qt, qtt = ellipse_factor(0.4)
        y0, y0t, y0tt = -0.3 * u, -0.3 * du, -0.3 * ddu
        r = np.stack([pf * cp, y0 + qf * sp, ct + z], -1)
        rt = np.stack([pt * cp, y0t + qt * sp, -st + z], -1)
        rth = np.stack([-pf * sp, qf * cp, z], -1)
        rtt = np.stack([ptt * cp, y0tt + qtt * sp, -ct + z], -1)
        rtth = np.stack([-pt * sp, qt * cp, z], -1)
        rthth = np.stack([-pf * cp, -qf * sp, z], -1)
        return r, rt, rth, rtt, rtth, rthth
    if surface["kind"] == "fourier_torus":
        w = surface["R"] + z
        wt = z.copy(); wth = z.copy(); wtt = z.copy(); wtth = z.copy(); wthth = z.copy()
        zt_ = z.copy(); zh = z.copy(); ztt = z.copy(); zth = z.copy(); zhh = z.copy(); zeta = z.copy()
        for cc, m, n in surface["terms"]:
            ph = m * th + n * t
            cph, sph = np.cos(ph), np.sin(ph)
            w = w + cc * cph
            wt = wt - cc * n * sph
            wth = wth - cc * m * sph
            wtt = wtt - cc * n * n * cph
            wtth = wtth - cc * m * n * cph
            wthth = wthth - cc * m * m * cph
            zeta = zeta + cc * sph
            zt_ = zt_ + cc * n * cph
            zh = zh + cc * m * cph
            ztt = ztt - cc * n * n * sph
            zth = zth - cc * m * n * sph
            zhh = zhh - cc * m * m * sph
        r = np.stack([w * ct, w * st, zeta], -1)
        rt = np.stack([wt * ct - w * st, wt * st + w * ct, zt_], -1)
        rth = np.stack([wth * ct, wth * st, zh], -1)
        rtt = np.stack([wtt * ct - 2 * wt * st - w * ct, wtt * st + 2 * wt * ct - w * st, ztt], -1)
        rtth = np.stack([wtth * ct - wth * st, wtth * st + wth * ct, zth], -1)
        rthth = np.stack([wthth * ct, wthth * st, zhh], -1)
        return r, rt, rth, rtt, rtth, rthth
    if surface["kind"] == "torus":
        a, b, c = surface["a"], surface["b"], surface["c"]
        m, eps = float(surface["m"]), surface["eps"]
        smt, cmt = np.sin(m * t), np.cos(m * t)
        w = surface["R"] + cp + eps * cmt
        wt, wth = -eps * m * smt + z, -sp
        wtt, wthth = -eps * m * m * cmt + z, -cp
        r = np.stack([a * w * ct, b * w * st, c * sp], -1)
        rt = np.stack([a * (wt * ct - w * st), b * (wt * st + w * ct), z], -1)
        rth = np.stack([a * wth * ct, b * wth * st, c * cp], -1)
        rtt = np.stack([a * (wtt * ct - 2 * wt * st - w * ct), b * (wtt * st + 2 * wt * ct - w * st), z], -1)
        rtth = np.stack([-a * wth * st, b * wth * ct, z], -1)
        rthth = np.stack([a * wthth * ct, b * wthth * st, -c * sp], -1)
        return r, rt, rth, rtt, rtth, rthth
    raise ValueError("unknown surface kind %r" % surface["kind"])


def normal_and_jacobian(surface, t, th):
    """Outward unit normal nu and J = |r_t x r_th| (assumption (iii), Section 2)."""
    _, rt, rth, _, _, _ = evaluate(surface, t, th)
    n = np.cross(rt, rth)
    J = np.sqrt(np.sum(n * n, -1))
    return n / J[..., None], J


_GL16_X, _GL16_W = np.polynomial.legendre.leggauss(16)
_LAM = (_GL16_X + 1) / 2          # Gauss-Legendre nodes on [0, 1]
_LAMW = _GL16_W / 2


def wrap_angle(d):
    """Map an angle difference to (-pi, pi] (real part for complex input)."""
    d = np.asarray(d)
    re = np.real(d)
    shift = np.round(re / (2 * np.pi)) * 2 * np.pi
    return d - shift


def difference(surface, t_s, th_s, t, th, stable):
    """r(t_s, th_s) - r(t, th).

    Where ``stable`` is true the difference is the line integral of the
    first derivatives along the straight parameter path (Section 4, Remark
    on cancellation): r(v) - r(u) = -int_0^1 Dr(gamma(lam)) [u - v] dlam,
    gamma = v + lam (u - v), with 16-point Gauss-Legendre.  Elsewhere it is
    the plain subtraction.  theta differences are wrapped to (-pi, pi].
    """
    t_s, th_s, t, th = np.broadcast_arrays(np.asarray(t_s, float), np.asarray(th_s), np.asarray(t, float), np.asarray(th))
    stable = np.broadcast_to(stable, t_s.shape)
    r_s = evaluate(surface, t_s, th_s)[0]
    r_0 = evaluate(surface, t, th)[0]
    out = r_s - r_0
    if np.any(stable):
        idx = np.nonzero(stable)
        ts, hs, tt, ht = t_s[idx], th_s[idx], t[idx], th[idx]
        dt = tt - ts
        dth = wrap_angle(ht - hs)
        acc = np.zeros(ts.shape + (3,), dtype=np.result_type(hs, ht, complex if np.iscomplexobj(hs) else float))
        for lam, w in zip(_LAM, _LAMW):
            _, rt, rth, _, _, _ = evaluate(surface, ts + lam * dt, hs + lam * dth)
            acc = acc + w * (rt * dt[..., None] + rth * dth[..., None])
        out = out.astype(acc.dtype)
        out[idx] = -acc
    return out


def tau0_stable(surface, t_s, th_s, t, th):
    """tau_0 = nu(v) . (r(v) - r(u)) by the second-derivative line integral
    of Section 4 (Remark): int_0^1 (lam - 1) nu(v) . D^2 r(gamma(lam))[delta, delta] dlam."""
    t_s, th_s, t, th = np.broadcast_arrays(np.asarray(t_s, float), np.asarray(th_s, float), np.asarray(t, float), np.asarray(th, float))
    nu, _ = normal_and_jacobian(surface, t_s, th_s)
    dt = t - t_s
    dth = wrap_angle(th - th_s)
    acc = np.zeros(t_s.shape)
    for lam, w in zip(_LAM, _LAMW):
        _, _, _, rtt, rtth, rthth = evaluate(surface, t_s + lam * dt, th_s + lam * dth)
        quad = rtt * (dt * dt)[..., None] + 2 * rtth * (dt * dth)[..., None] + rthth * (dth * dth)[..., None]
        acc = acc + w * (lam - 1) * np.sum(nu * quad, -1)
    return acc
