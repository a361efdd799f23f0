"""Closed forms for charges inside a dielectric sphere (pins for the oracle).

These are independent of the boundary-element discretisation: they solve the
mixed-dielectric Poisson problem of Sec. 2.1 exactly for a sphere of radius a
by separation of variables.  With the interior-limit reading of Eq. ASC the
operator K' has eigenvalue -1/(2(2l+1)) on degree-l spherical harmonics, so
the same series also gives the exact BIBEE energies on a sphere (Eq. CFA with
lambda in {-1/2, 0}).

    dG = -1/2 * 332.0637 * sum_ij q_i q_j / a * sum_l f_l (r_i r_j / a^2)^l P_l(cos t_ij)

    full solve (Kirkwood 1934): f_l = (l+1)(eps_out-eps_in) / (eps_in((l+1) eps_out + l eps_in))
    BIBEE/CFA  (lambda = -1/2):  f_l = (l+1)/(2l+1) * (1/eps_in - 1/eps_out)
    BIBEE/P    (lambda = 0):     f_l = (l+1)/(2l+1) * 2 (eps_out-eps_in)/(eps_in (eps_in+eps_out))

The l = 0 term with one central charge is the Born energy
    dG_Born = -1/2 * 332.0637 q^2 / a * (1/eps_in - 1/eps_out).
"""
import numpy as np

KCAL = 332.0637


def born_energy(q, a, eps_in, eps_out):
    return -0.5 * KCAL * q * q / a * (1.0 / eps_in - 1.0 / eps_out)


def _factor(l, eps_in, eps_out, kind):
    l = np.asarray(l, dtype=np.float64)
    if kind == "full":
        return (l + 1) * (eps_out - eps_in) / (eps_in * ((l + 1) * eps_out + l * eps_in))
    if kind == "cfa":
        return (l + 1) / (2 * l + 1) * (1.0 / eps_in - 1.0 / eps_out)
    if kind == "p":
        return (l + 1) / (2 * l + 1) * 2.0 * (eps_out - eps_in) / (eps_in * (eps_in + eps_out))
    raise ValueError(kind)


def sphere_energy(charges, a, eps_in, eps_out, kind="full", center=(0, 0, 0), tol=1e-17,
                  lmax=2000):
    """Series energy (kcal/mol) of point charges inside a sphere of radius a."""
    ch = np.asarray(charges, dtype=np.float64)
    x = ch[:, :3] - np.asarray(center, dtype=np.float64)
    q = ch[:, 3]
    r = np.linalg.norm(x, axis=1)
    rr = np.outer(r, r)
    with np.errstate(invalid="ignore", divide="ignore"):
        cos = (x @ x.T) / rr
    cos = np.where(rr > 0, np.clip(cos, -1.0, 1.0), 1.0)
    t = rr / (a * a)
    qq = np.outer(q, q)
    total = 0.0
    p_prev = np.ones_like(cos)       # P_0
    p_cur = cos.copy()               # P_1
    tl = np.ones_like(t)             # t^l
    for l in range(lmax + 1):
        if l == 0:
            pl = p_prev
        elif l == 1:
            pl = p_cur
        else:
            p_next = ((2 * l - 1) * cos * p_cur - (l - 1) * p_prev) / l
            p_prev, p_cur = p_cur, p_next
            pl = p_cur
        term = _factor(l, eps_in, eps_out, kind) * float(np.sum(qq * tl * pl))
        total += term
        if l > 2 and np.max(np.abs(qq) * tl) * _factor(l, eps_in, eps_out, kind) < tol * max(abs(total), 1e-300):
            break
        tl = tl * t
    return -0.5 * KCAL / a * total
