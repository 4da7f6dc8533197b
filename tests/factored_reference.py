"""The paper's factored evaluation of the four responses, in its own notation.

This is a test-side pin for the oracle, not an oracle: it never reads the
oracle's Eq. (3) tables.  It starts from the generalised weights (a, b, m, n) of
Eq. (5) and follows Section 4.3 step by step:

* K_x: horizontal difference F (Eq. 6) per row, vertical smoothing (Eq. 7).
* K_y: "the same manner, using different coefficients" -- horizontal smoothing
  a*[1, n, m, n, 1], vertical difference [-1, -b, 0, b, 1].
* K_d+ = K_d + K_dt: row convolutions F_k0, F_k1 (Eq. 12) and the reuse
  F_k3 = -F_k1, F_k4 = -F_k0 (Eq. 14) combined as in Eq. (15).
* K_d- = K_d - K_dt: either directly (Eq. 16, Eq. 17) or through the
  decomposition of Eq. (18) into the K_x row result F and the column
  difference D (Eq. 19).
* G_d = (G_d+ + G_d-)/2 and G_dt = (G_d+ - G_d-)/2 (Eq. 11).

Only the valid interior (2 <= y <= H-3, 2 <= x <= W-3) is produced; it is
returned as int64 planes of shape (H-4, W-4).
"""
from __future__ import annotations

import numpy as np


def _taps(img: np.ndarray):
    """p^0..p^4 of every row: the five pixels at columns x-2..x+2 (x interior)."""
    I = img.astype(np.int64)
    W = I.shape[1]
    return [I[:, j:W - 4 + j] for j in range(5)]


def _vertical(F, w):
    """sum_t w[t] * F^{v-2+t} for every interior centre row v."""
    H = F.shape[0]
    return sum(w[t] * F[t:H - 4 + t] for t in range(5))


def factored_responses(img: np.ndarray, a=1, b=2, m=6, n=4, kd_minus="eq19"):
    p0, p1, p2, p3, p4 = _taps(img)

    # K_x: Eq. (6) then Eq. (7).
    F = -1 * p0 + (-b) * p1 + b * p3 + p4
    Gx = _vertical(F, [a, a * n, a * m, a * n, a])

    # K_y: horizontal smoothing, vertical difference.
    Fy = a * (p0 + n * p1 + m * p2 + n * p3 + p4)
    Gy = _vertical(Fy, [-1, -b, 0, b, 1])

    # K_d+: Eq. (12), Eq. (14), Eq. (15).
    Fk0 = -a * m * p0 + a * (-n - b) * p1 + (-2 * a) * p2 + a * (-n - b) * p3 + (-a * m) * p4
    Fk1 = a * (b - n) * p0 + (-a * m * b) * p1 + (-2 * a * n * b) * p2 + (-a * m * b) * p3 \
        + a * (b - n) * p4
    H = Fk0.shape[0]
    Gdp = Fk0[0:H - 4] + Fk1[1:H - 3] - Fk1[3:H - 1] - Fk0[4:H]

    if kd_minus == "eq17":
        # K_d-: Eq. (16), Eq. (17).
        Gk0 = -a * m * p0 + a * (b - n) * p1 + a * (n - b) * p3 + a * m * p4
        Gk1 = a * (-n - b) * p0 + (-a * m * b) * p1 + (a * m * b) * p3 + a * (n + b) * p4
        Gk2 = (-2 * a) * p0 + (-2 * a * n * b) * p1 + (2 * a * n * b) * p3 + (2 * a) * p4
        Gdm = Gk0[0:H - 4] + Gk1[1:H - 3] + Gk2[2:H - 2] + Gk1[3:H - 1] + Gk0[4:H]
    else:
        # K_d-: Eq. (18), Eq. (19) -- reuse F of K_x plus D = p3 - p1.
        D = -p1 + p3
        Gdm = _vertical(F, [a * m, a * (n + b), 2 * a, a * (n + b), a * m]) \
            - _vertical(D, [a * (m * b + b - n), a * (n * b + b * b - m * b), a * (2 * b - 2 * n * b),
                            a * (n * b + b * b - m * b), a * (m * b - n + b)])

    # Eq. (11): both sums are even, so the halving is exact.
    assert np.all((Gdp + Gdm) % 2 == 0)
    Gd = (Gdp + Gdm) // 2
    Gdt = (Gdp - Gdm) // 2
    return np.stack([Gx, Gy, Gd, Gdt])
