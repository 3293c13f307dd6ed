"""Offline generator of the 16-node generalized Gaussian quadrature (GGQ) tables.

The method (Section 3.1, Eq. (S123)) integrates the t_s-direction over the
self panel and the two adjacent panels of a target node t_j^l with 16-node
rules whose nodes and weights depend on the target index l, and which are
exact (to ~1e-14) on the functions that appear after the azimuthal
integration (Theorem "thm:logsing"): p(s) + q(s) log|s - tau| with p, q
polynomials of degree < 16.  The paper takes its rules from an external GGQ
code that is not available here, so this script builds its own rules with
the usual generalized-Gaussian recipe:

  1. an oversampled composite Gauss-Legendre rule, graded dyadically toward
     the singular point tau (or toward the panel end nearest to it);
  2. an SVD of the 32 functions {P_n, P_n log|s - tau|}, n < 16, sampled
     with the square roots of those weights (orthogonal directions of the
     function class, each scaled by its singular value);
  3. an interpolatory start rule whose nodes are picked by pivoted QR;
  4. node elimination: drop the least significant node and restore
     exactness by min-norm Gauss-Newton on (nodes, weights), until 16 nodes
     remain.

Rules are built on the reference panel [-1, 1].  Target positions tau, in
the coordinates of the source panel:
  * self panel (delta = 0):          tau = x_l           (x_l Legendre node)
  * source panel left of target:     tau = x_l + 2       (delta = -1)
  * source panel right of target:    tau = x_l - 2       (delta = +1)
The delta = +1 and the self rules for l < 8 are mirror images (s -> -s) of
the delta = -1 rule for 15 - l and of the self rule for 15 - l.

Output: ggq16.txt next to this file.  Run:  python gen_ggq.py
"""
import os
import sys
import numpy as np
import scipy.linalg as sla

NQ = 16
XL, WL = np.polynomial.legendre.leggauss(NQ)


def _legendre_and_derivative(x, nmax):
    x = np.asarray(x, float)
    P = np.zeros((nmax,) + x.shape)
    dP = np.zeros_like(P)
    P[0] = 1.0
    P[1] = x
    dP[1] = 1.0
    for n in range(1, nmax - 1):
        P[n + 1] = ((2 * n + 1) * x * P[n] - n * P[n - 1]) / (n + 1)
        dP[n + 1] = dP[n - 1] + (2 * n + 1) * P[n]
    return P, dP


def _class_functions(x, tau):
    """The 32 functions P_n(s), P_n(s) log|s - tau| and their s-derivatives."""
    P, dP = _legendre_and_derivative(x, NQ)
    L = np.log(np.abs(x - tau))
    dL = 1.0 / (x - tau)
    return np.vstack([P, P * L]), np.vstack([dP, dP * L + P * dL])


def _oversampled_rule(tau):
    xs, ws = [], []

    def panel(a, b):
        xs.append((a + b) / 2 + (b - a) / 2 * XL)
        ws.append((b - a) / 2 * WL)

    def graded(a, b, toward_a):
        length = b - a
        cuts, d = [], length
        while d > 2e-13:
            d /= 2
            cuts.append(d)
        edges = sorted(set([0.0] + cuts + [length]))
        for e0, e1 in zip(edges[:-1], edges[1:]):
            if toward_a:
                panel(a + e0, a + e1)
            else:
                panel(b - e1, b - e0)

    if -1.0 < tau < 1.0:
        graded(-1.0, tau, False)
        graded(tau, 1.0, True)
    else:
        dist = min(abs(tau - 1.0), abs(tau + 1.0))
        a, b = -1.0, 1.0
        while (b - a) > dist / 2 and (b - a) > 1e-3:
            m = (a + b) / 2
            if tau > 1.0:
                panel(a, m)
                a = m
            else:
                panel(m, b)
                b = m
        panel(a, b)
    return np.concatenate(xs), np.concatenate(ws)


def build_rule(tau, tol=1e-13, prefer_positive=True):
    X, W = _oversampled_rule(tau)
    F, _ = _class_functions(X, tau)
    mom_phi = F @ W
    U, S, _ = np.linalg.svd(F * np.sqrt(W)[None, :], full_matrices=False)
    C = U.T
    mom = C @ mom_phi

    def G(x):
        f, df = _class_functions(x, tau)
        return C @ f, C @ df

    rank = int(np.sum(S > 1e-15 * S[0]))
    Ux = ((C / S[:, None]) @ F) * np.sqrt(W)[None, :]
    _, _, piv = sla.qr(Ux[:rank], pivoting=True, mode="economic")
    x = X[np.sort(piv[:rank])]
    g, _ = G(x)
    w = np.linalg.lstsq(g, mom, rcond=None)[0]

    def gauss_newton(x, w, iters=80):
        n = len(w)
        g, dg = G(x)
        R = g @ w - mom
        nr = np.linalg.norm(R)
        for _ in range(iters):
            J = np.hstack([g, dg * w[None, :]])
            d = np.linalg.pinv(J, rcond=1e-12) @ (-R)
            lam, accepted = 1.0, False
            while lam > 1e-9:
                xn = x + lam * d[n:]
                wn = w + lam * d[:n]
                if np.all(np.abs(xn) < 1) and np.all(xn != tau):
                    gn, dgn = G(xn)
                    Rn = gn @ wn - mom
                    nrn = np.linalg.norm(Rn)
                    if nrn < nr:
                        accepted = True
                        break
                lam /= 2
            if not accepted:
                break
            x, w, g, dg, R, nr = xn, wn, gn, dgn, Rn, nrn
            if nr < 1e-16:
                break
        return x, w, nr

    x, w, _ = gauss_newton(x, w)
    while len(x) > NQ:
        g, _ = G(x)
        significance = np.abs(w) * np.sum(g ** 2, axis=0)
        chosen = fallback = None
        for j in np.argsort(significance):
            keep = np.ones(len(x), bool)
            keep[j] = False
            x2, w2, r2 = gauss_newton(x[keep].copy(), w[keep].copy())
            if r2 >= tol:
                continue
            if np.all(w2 > 0) or not prefer_positive:
                chosen = (x2, w2)
                break
            if fallback is None:
                fallback = (x2, w2)
        chosen = chosen or fallback
        if chosen is None:
            return None
        order = np.argsort(chosen[0])
        x, w = chosen[0][order], chosen[1][order]
    x, w, _ = gauss_newton(x, w, iters=200)
    f, _ = _class_functions(x, tau)
    err = float(np.max(np.abs(f @ w - mom_phi)))
    order = np.argsort(x)
    return x[order], w[order], err


def main(path=None):
    path = path or os.path.join(os.path.dirname(os.path.abspath(__file__)), "ggq16.txt")
    rules = {}
    for l in range(NQ // 2, NQ):
        out = build_rule(XL[l])
        if out is None:
            raise RuntimeError("self rule for l=%d did not converge" % l)
        rules[(0, l)] = out
        x, w, e = out
        rules[(0, NQ - 1 - l)] = (-x[::-1], w[::-1], e)
    for l in range(NQ):
        out = build_rule(XL[l] + 2.0)
        if out is None:
            raise RuntimeError("adjacent rule for l=%d did not converge" % l)
        rules[(-1, l)] = out
    for l in range(NQ):
        x, w, e = rules[(-1, NQ - 1 - l)]
        rules[(1, l)] = (-x[::-1], w[::-1], e)
    with open(path, "w") as fh:
        fh.write("# 16-node generalized Gaussian rules on the reference panel [-1,1]\n")
        fh.write("# exact (to the listed error) for P_n(s) and P_n(s) log|s-tau|, n<16\n")
        fh.write("# line format: delta l err x_1..x_16 w_1..w_16\n")
        fh.write("# delta: -1 source panel left of the target panel (tau = x_l + 2),\n")
        fh.write("#         0 self panel (tau = x_l), +1 source panel right (tau = x_l - 2)\n")
        for delta in (-1, 0, 1):
            for l in range(NQ):
                x, w, e = rules[(delta, l)]
                fh.write("%d %d %.3e " % (delta, l, e))
                fh.write(" ".join("%.17e" % v for v in x) + " ")
                fh.write(" ".join("%.17e" % v for v in w) + "\n")
                print("delta %+d l %2d err %.2e min w %.3e" % (delta, l, e, w.min()))
    return path


if __name__ == "__main__":
    main(sys.argv[1] if len(sys.argv) > 1 else None)
