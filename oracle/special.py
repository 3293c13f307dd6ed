"""Oracle: special functions of the singularity-swapping step (Sections 3.3 and 4).

TEST INFRASTRUCTURE ONLY.  Plain FP64 numpy, scalar-per-pair loops are
vectorised over a batch of parameters b.

  ellipke(m, m1)       complete elliptic integrals K, E by the arithmetic-
                       geometric mean (DLMF 19.8.1, 19.8.6); m1 = 1 - m is
                       passed separately to keep it accurate near m = 1.
  a_modes(b, L)        A_m(b) = <s_{0,b}^{-1/2}>_m, m = 0..L  (Eq. (Am)),
                       normalised by the closed form A_0 = (2/pi) K(e^{-2b}).
                       If L*b <= 7 the paper's difference recurrence
                       (Eq. (diff-recurrence)) runs forward from A_0 and
                       D_1 = A_1 - A_0 (A_1 = 2/(pi q) (K - E), q = e^{-b});
                       otherwise Miller's backward recurrence runs on the
                       ratios A_{m-1}/A_m = 1 + delta_m, written for delta_m
                       so that the differences D_m = -A_m delta_m come out
                       without cancellation.
  b_modes(b, A, D)     B_m(0,b) = <s_{0,b}^{-3/2}>_m, m = 0..L, by the two-
                       term closed form -(m - 1/2) e^b (cosh b A_m - A_{m-1})
                       / sinh^2 b (from Eq. (Am-Q) and the Legendre
                       derivative identity), with A_{-1} = A_1.  The paper's
                       forward recurrence (Eq. (Bm-recurrence)) loses
                       accuracy like e^{2mb}, so it is used only as a pin.
"""
import numpy as np

FORWARD_LIMIT = 7.0      # use the forward difference recurrence when L*b <= this
MILLER_EPS_LOG = 39.2    # ln(1e17): Miller start N = L + ceil(MILLER_EPS_LOG/(2b)) + 16


def ellipke(m, m1):
    """K(m), E(m) (parameter m, m1 = 1 - m) by the AGM, DLMF 19.8."""
    m = np.asarray(m, float)
    a = np.ones_like(m)
    g = np.sqrt(np.asarray(m1, float))
    c2sum = 0.5 * m                      # 2^{n-1} c_n^2 summed, c_0^2 = m
    scale = 0.5
    for _ in range(40):
        an = 0.5 * (a + g)
        cn = 0.5 * (a - g)
        g = np.sqrt(a * g)
        a = an
        scale *= 2.0
        c2sum = c2sum + scale * cn * cn
        if np.all(np.abs(cn) <= 1e-17 * a):
            break
    K = np.pi / (2 * a)
    E = K * (1.0 - c2sum)
    return K, E


def a0_a1(b):
    """Closed forms A_0 = (2/pi) K(q^2), A_1 = (2/(pi q)) (K(q^2) - E(q^2)), q = e^{-b}."""
    b = np.asarray(b, float)
    q = np.exp(-b)
    K, E = ellipke(q * q, -np.expm1(-2 * b))
    return 2 / np.pi * K, 2 / (np.pi * q) * (K - E), K, E


def a_modes(b, L):
    """A_m(b) and D_m = A_m - A_{m-1} for m = 0..L (D_0 := A_0 - A_1).

    b: array of shape (B,).  Returns A, D of shape (B, L+1).
    """
    b = np.atleast_1d(np.asarray(b, float))
    B = b.shape[0]
    A = np.zeros((B, L + 1))
    D = np.zeros((B, L + 1))
    A0, A1, K, E = a0_a1(b)
    q = np.exp(-b)
    sh2 = np.sinh(b / 2) ** 2
    ch = np.cosh(b)
    forward = L * b <= FORWARD_LIMIT
    # forward difference recurrence (Eq. (diff-recurrence))
    if np.any(forward):
        i = np.nonzero(forward)[0]
        a_m = A0[i].copy()
        d_m = (2 / np.pi) * ((K[i] - E[i]) / q[i] - K[i])      # D_1 = A_1 - A_0
        A[i, 0] = a_m
        D[i, 0] = -d_m
        if L >= 1:
            a_m = a_m + d_m
            A[i, 1] = a_m
            D[i, 1] = d_m
        for m in range(1, L):
            d_m = ((2 * m - 1) * d_m + 8 * m * sh2[i] * a_m) / (2 * m + 1)
            a_m = a_m + d_m
            A[i, m + 1] = a_m
            D[i, m + 1] = d_m
    # Miller backward recurrence on delta_m = A_{m-1}/A_m - 1
    if np.any(~forward):
        for i in np.nonzero(~forward)[0]:
            bi = b[i]
            N = L + int(np.ceil(MILLER_EPS_LOG / (2 * bi))) + 16
            delta = np.zeros(N + 2)
            # A_{N+1} = 0 gives rho_N = 4N cosh b / (2N - 1)
            delta[N] = (2 * N + 1 + 8 * N * sh2[i]) / (2 * N - 1)
            for m in range(N - 1, 0, -1):
                dn = delta[m + 1]
                delta[m] = (8 * m * sh2[i] + (2 * m + 1) * dn / (1 + dn)) / (2 * m - 1)
            a_m = A0[i]
            A[i, 0] = a_m
            for m in range(1, L + 1):
                a_new = a_m / (1 + delta[m])
                D[i, m] = -a_new * delta[m]
                a_m = a_new
                A[i, m] = a_m
            D[i, 0] = -D[i, 1] if L >= 1 else A0[i] - A1[i]
    return A, D


def b_modes(b, A, D):
    """B_m(0, b) for m = 0..L from A_m and D_m (two-term closed form)."""
    b = np.atleast_1d(np.asarray(b, float))
    L = A.shape[1] - 1
    m = np.arange(L + 1)[None, :]
    sh2h = (np.sinh(b / 2) ** 2)[:, None]
    # cosh b A_m - A_{m-1} = D_m + 2 sinh^2(b/2) A_m, with A_{-1} = A_1 (D_0 = A_0 - A_1)
    core = D + 2 * sh2h * A
    return -(m - 0.5) * np.exp(b)[:, None] * core / (np.sinh(b) ** 2)[:, None]


def b0_closed_form(b):
    """B_0 = 4E(e^{-2b}) / (pi (1 - e^{-2b})^2) - A_0 / (1 - e^{-2b})   (Eq. (B0))."""
    A0, _, K, E = a0_a1(b)
    om = -np.expm1(-2 * np.asarray(b, float))
    return 4 * E / (np.pi * om * om) - A0 / om
