"""LDA exchange-correlation (oracle; test infrastructure).

Sec. 3.1 of the paper:
  exchange (Kohn-Sham/Slater):  E_x = -(3/4)(3/pi)^(1/3) int rho^(4/3),
                                V_x = -(3 rho/pi)^(1/3)                 (Sec. 3.1)
  correlation (Perdew-Zunger), r_s = (3/(4 pi rho))^(1/3):
    eps_c = A ln r_s + B + C r_s ln r_s + D r_s          if r_s < 1
          = gamma / (1 + beta1 sqrt(r_s) + beta2 r_s)    if r_s >= 1
    V_c   = A ln r_s + (B - A/3) + (2/3) C r_s ln r_s + (1/3)(2D - C) r_s      if r_s < 1
          = eps_c (1 + (7/6) beta1 sqrt(r_s) + (4/3) beta2 r_s)
                  / (1 + beta1 sqrt(r_s) + beta2 r_s)                          if r_s >= 1
                                                                               (Sec. 3.1)
  constants A=0.0311, B=-0.048, gamma=-0.1423, beta1=1.0529, beta2=0.3334,
  C=0.0020, D=-0.0116.
The exchange energy per electron is eps_x = -(3/4)(3/pi)^(1/3) rho^(1/3), so
E_xc = int rho (eps_x + eps_c).

Readings: r_s = 1 takes the r_s >= 1 branch, as printed; rho <= 1e-30 (and
negative rho, which a mixed density can reach) gives eps = V = 0.
"""
import numpy as np

A = 0.0311
B = -0.048
GAMMA = -0.1423
BETA1 = 1.0529
BETA2 = 0.3334
C = 0.0020
D = -0.0116
RHO_MIN = 1e-30


def lda(rho):
    """Return (eps_xc, v_xc) at each density value (arrays of rho's shape)."""
    rho = np.asarray(rho, dtype=np.float64)
    eps = np.zeros_like(rho)
    v = np.zeros_like(rho)
    m = rho > RHO_MIN
    r = rho[m]
    eps_x = -0.75 * (3.0 / np.pi) ** (1.0 / 3.0) * r ** (1.0 / 3.0)
    v_x = -(3.0 * r / np.pi) ** (1.0 / 3.0)
    rs = (3.0 / (4.0 * np.pi * r)) ** (1.0 / 3.0)
    lo = rs < 1.0
    eps_c = np.empty_like(r)
    v_c = np.empty_like(r)
    rl = rs[lo]
    ln = np.log(rl)
    eps_c[lo] = A * ln + B + C * rl * ln + D * rl
    v_c[lo] = A * ln + (B - A / 3.0) + (2.0 / 3.0) * C * rl * ln + (1.0 / 3.0) * (2.0 * D - C) * rl
    rh = rs[~lo]
    sq = np.sqrt(rh)
    den = 1.0 + BETA1 * sq + BETA2 * rh
    e_hi = GAMMA / den
    eps_c[~lo] = e_hi
    v_c[~lo] = e_hi * (1.0 + (7.0 / 6.0) * BETA1 * sq + (4.0 / 3.0) * BETA2 * rh) / den
    eps[m] = eps_x + eps_c
    v[m] = v_x + v_c
    return eps, v
