"""FP64 CPU oracle for the FMM-BEM solvation model (arXiv:1007.4591).

TEST INFRASTRUCTURE ONLY: the plain dense O(n^2) reference that the CUDA path
is checked against.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline leg may import it; the product package never does.

What it computes (Sec. 2.1-2.2 of the paper, in the reading fixed below):

* Eq. ASC with the interior limit of the normal derivative, which gives the
  second-kind system  (I + Ehat K') sigma = -Ehat * (B q),
  Ehat = 2 (eps_in - eps_out) / (eps_in + eps_out).  sigma is eps_in times
  the physical induced surface charge (the paper's Eq. ASC omits the 1/eps_in
  of the Poisson source term), so the reaction potential is C sigma / eps_in.
* Eq. reac and the solvation energy  dG = 1/2 sum_k q_k phi_reac(x_k), in
  kcal/mol with 332.0637 kcal A / (mol e^2) and G = 1/(4 pi r):
  dG = 4 pi * 332.0637 / (2 eps_in) * q . (C sigma).
* Eq. CFA and its variants (Sec. 2.2): K' replaced by lambda * I,
  sigma_hat = -Ehat / (1 + Ehat lambda) * (B q), lambda in {-1/2, 0, +1/2}.
* The matrix form A x = B q, phi = C x of Sec. 2.1 and its adjoint, giving
  d dG / d q_k and d dG / d x_k (solve A^T lam = C^T q).
* Restarted GMRES (Saad & Schultz 1986) with modified Gram-Schmidt Arnoldi
  and Givens rotations, x0 = 0, relative residual |b - A x| / |b|.
* The higher-accuracy panel integration (Sec. 2.1 names exact integrals over
  flat panels as the alternative to quadrature): with exact_charge_near, the
  charge-panel pairs of C, C^T and grad C closer than 2.5 sqrt(A_j) take the
  exact single-layer integral over the flat panel.

The dense sums live in ``bem_oracle.c`` (compiled with gcc, OpenMP over
targets); this module does the linear algebra around them in numpy.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import numpy as np

KCAL_PER_MOL = 332.0637          # e^2 / (4 pi eps0 A) in kcal/mol
_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "bem_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

BIBEE_LAMBDA = {"cfa": -0.5, "p": 0.0, "plus_half": 0.5}


def build(force: bool = False) -> str:
    """Compile the C oracle (gcc, OpenMP, no fused multiply-add contraction)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fPIC", "-shared",
               "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        d = ctypes.POINTER(ctypes.c_double)
        i64 = ctypes.c_int64
        ci = ctypes.c_int
        sig = {
            "oracle_quad_rule": (ci, [ci, d, d]),
            "oracle_geometry": (ci, [d, i64, ci, d, d, d, d, d]),
            "oracle_kprime": (None, [i64, ci, d, d, d, d, d, d]),
            "oracle_kprime_rows": (None, [i64, ci, d, d, d, d, d, i64,
                                          ctypes.POINTER(ctypes.c_int64), d]),
            "oracle_kprime_t": (None, [i64, ci, d, d, d, d, d, d]),
            "oracle_kprime_dense": (None, [i64, ci, d, d, d, d, d]),
            "oracle_bq": (None, [i64, d, d, i64, d, d, d]),
            "oracle_bt": (None, [i64, d, d, i64, d, d, d]),
            "oracle_c": (None, [i64, ci, d, d, i64, d, d, d]),
            "oracle_ct": (None, [i64, ci, d, d, i64, d, d, d]),
            "oracle_grad_c": (None, [i64, ci, d, d, i64, d, d, d]),
            "oracle_grad_bt": (None, [i64, d, d, i64, d, d, d]),
            "oracle_solid_angle": (ctypes.c_double, [d, d]),
            "oracle_panel_dn": (ctypes.c_double, [d, d, d]),
            "oracle_panel_phi": (ctypes.c_double, [d, d]),
            "oracle_panel_grad_phi": (None, [d, d, d]),
            "oracle_c_exact": (None, [i64, ci, d, d, d, d, d, i64, d, d, d]),
            "oracle_ct_exact": (None, [i64, ci, d, d, d, d, d, i64, d, d, d]),
            "oracle_grad_c_exact": (None, [i64, ci, d, d, d, d, d, i64, d, d, d]),
            "oracle_kprime_rows_near_exact": (None, [i64, ci, d, d, d, d, d, d, d, i64,
                                                     ctypes.POINTER(ctypes.c_int64), d]),
            "oracle_kprime_rows_galerkin": (None, [i64, ci, d, d, d, d, d, d, d, i64,
                                                   ctypes.POINTER(ctypes.c_int64), d]),
            "oracle_bq_galerkin": (None, [i64, ci, d, d, d, d, i64, d, d, d]),
            "oracle_kprime_t_galerkin": (None, [i64, ci, d, d, d, d, d, d, d, d]),
            "oracle_bt_galerkin": (None, [i64, ci, d, d, d, d, i64, d, d, d, d]),
            "oracle_num_threads": (ci, []),
            "oracle_set_threads": (None, [ci]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
    return _lib


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _c(a, dtype=np.float64):
    return np.ascontiguousarray(a, dtype=dtype)


def num_threads() -> int:
    return int(_load().oracle_num_threads())


def set_threads(t: int) -> None:
    _load().oracle_set_threads(int(t))


def quad_rule(nq: int = 7):
    """Barycentric points [nq, 3] and weights [nq] of the triangle rule."""
    bary = np.zeros((nq, 3))
    w = np.zeros(nq)
    if _load().oracle_quad_rule(nq, _p(bary), _p(w)) != 0:
        raise ValueError("nq must be 1 or 7")
    return bary, w


def ehat(eps_in: float, eps_out: float) -> float:
    """Ehat = 2 (eps_in - eps_out) / (eps_in + eps_out): A = I + Ehat K'."""
    return 2.0 * (eps_in - eps_out) / (eps_in + eps_out)


def bibee_factor(eps_in: float, eps_out: float, lam: float) -> float:
    """sigma_hat = bibee_factor * (B q): K' replaced by lam * I in the ASC system."""
    e = ehat(eps_in, eps_out)
    return -e / (1.0 + e * lam)


def solid_angle(t, tri) -> float:
    """int_T h / R^3 dA: the solid angle of the flat triangle tri[3][3] seen
    from t, positive when t lies on the side its right-hand normal points to."""
    lib = _load()
    return float(lib.oracle_solid_angle(_p(_c(t)), _p(_c(tri))))


def panel_dn(t, n, tri) -> float:
    """int_T -(t - y).n / (4 pi |t - y|^3) dA_y, exactly, for a flat triangle."""
    lib = _load()
    return float(lib.oracle_panel_dn(_p(_c(t)), _p(_c(n)), _p(_c(tri))))


def panel_phi(t, tri) -> float:
    """int_T dA_y / (4 pi |t - y|), exactly, for a flat triangle (the
    single-layer potential of a unit density on one panel)."""
    lib = _load()
    return float(lib.oracle_panel_phi(_p(_c(t)), _p(_c(tri))))


def panel_grad_phi(t, tri):
    """grad_t of panel_phi: -int_T (t - y) / (4 pi |t - y|^3) dA_y."""
    g = np.empty(3)
    _load().oracle_panel_grad_phi(_p(_c(t)), _p(_c(tri)), _p(g))
    return g


def normal_field(targets, normals, charges):
    """Normal derivative of the charges' Coulomb potential at arbitrary points
    (the B q of Sec. 2.1 with the collocation points and normals replaced by
    any points and unit vectors):
    E_i = sum_k q_k [-(t_i - x_k).n_i] / (4 pi |t_i - x_k|^3).
    targets, normals [n, 3]; charges [nc, 4] (x, y, z, q)."""
    t = _c(targets).reshape(-1, 3)
    nv = _c(normals).reshape(-1, 3)
    ch = _c(charges).reshape(-1, 4)
    xq, q = _c(ch[:, :3]), _c(ch[:, 3])
    E = np.empty(t.shape[0])
    _load().oracle_bq(t.shape[0], _p(t), _p(nv), ch.shape[0], _p(xq), _p(q), _p(E))
    return E


class Problem:
    """Dense discrete operators of one molecule (panels + point charges)."""

    def __init__(self, panels, charges, eps_in: float, eps_out: float, nq: int = 7,
                 exact_charge_near: bool = False):
        """exact_charge_near: C, C^T and grad C integrate the charge-panel
        pairs closer than 2.5 sqrt(A_j) exactly over the flat panel (the
        higher-accuracy panel integration of Sec. 2.1), the rest by the rule."""
        lib = _load()
        self.exact_charge_near = bool(exact_charge_near)
        self.panels = _c(panels).reshape(-1, 3, 3)
        ch = _c(charges).reshape(-1, 4)
        self.xq = _c(ch[:, :3])
        self.q = _c(ch[:, 3])
        self.eps_in, self.eps_out, self.nq = float(eps_in), float(eps_out), int(nq)
        n = self.n = self.panels.shape[0]
        self.nc = self.xq.shape[0]
        self.cen = np.zeros((n, 3))
        self.nrm = np.zeros((n, 3))
        self.area = np.zeros(n)
        self.qp = np.zeros((n, nq, 3))
        self.qw = np.zeros((n, nq))
        rc = lib.oracle_geometry(_p(self.panels), n, nq, _p(self.cen), _p(self.nrm),
                                 _p(self.area), _p(self.qp), _p(self.qw))
        if rc != 0:
            raise ValueError(f"degenerate panel or bad rule (code {rc})")
        self.ehat = ehat(eps_in, eps_out)

    # --- operators (Sec. 2.1 matrix form) ---------------------------------
    def kprime(self, x):
        x = _c(x)
        y = np.empty(self.n)
        _load().oracle_kprime(self.n, self.nq, _p(self.cen), _p(self.nrm), _p(self.qp),
                              _p(self.qw), _p(x), _p(y))
        return y

    def kprime_rows(self, x, rows):
        x = _c(x)
        rows = _c(rows, np.int64)
        y = np.empty(rows.shape[0])
        _load().oracle_kprime_rows(self.n, self.nq, _p(self.cen), _p(self.nrm), _p(self.qp),
                                   _p(self.qw), _p(x), rows.shape[0],
                                   rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _p(y))
        return y

    def kprime_rows_near_exact(self, x, rows):
        """Rows of K' x with the exact flat-triangle integral for the
        near-singular pairs (|c_i - c_j| <= 2.5 sqrt(A_i)) and the quadrature
        rule for all other pairs."""
        x = _c(x)
        rows = _c(rows, np.int64)
        y = np.empty(rows.shape[0])
        _load().oracle_kprime_rows_near_exact(self.n, self.nq, _p(self.cen), _p(self.nrm), _p(self.area),
                                              _p(self.panels), _p(self.qp), _p(self.qw), _p(x),
                                              rows.shape[0],
                                              rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _p(y))
        return y

    def kprime_rows_galerkin(self, x, rows):
        """Rows of the Galerkin K' x: each row averaged over its panel by the
        rule, the near-singular inner integrals exact."""
        x = _c(x)
        rows = _c(rows, np.int64)
        y = np.empty(rows.shape[0])
        _load().oracle_kprime_rows_galerkin(self.n, self.nq, _p(self.cen), _p(self.nrm), _p(self.area),
                                            _p(self.panels), _p(self.qp), _p(self.qw), _p(x),
                                            rows.shape[0],
                                            rows.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _p(y))
        return y

    def kprime_galerkin(self, x):
        return self.kprime_rows_galerkin(x, np.arange(self.n))

    def bq_galerkin(self, q=None):
        """Normal field of the charges averaged over each panel by the rule."""
        q = self.q if q is None else _c(q)
        E = np.empty(self.n)
        _load().oracle_bq_galerkin(self.n, self.nq, _p(self.nrm), _p(self.area), _p(self.qp), _p(self.qw),
                                   self.nc, _p(self.xq), _p(q), _p(E))
        return E

    def solve_galerkin(self, tol: float = 1e-10, restart: int = 30, maxiter: int = 500,
                       transpose: bool = False, b=None):
        """sigma from (I + Ehat K'_G) sigma = -Ehat B_G q (Galerkin form), or
        with transpose the system (I + Ehat K'_G^T) x = b."""
        if transpose:
            op = lambda v: _c(v) + self.ehat * self.kprime_t_galerkin(v)
        else:
            op = lambda v: _c(v) + self.ehat * self.kprime_galerkin(v)
        b = -self.ehat * self.bq_galerkin() if b is None else _c(b)
        return gmres(op, b, tol=tol, restart=restart, maxiter=maxiter)

    def kprime_t_galerkin(self, x):
        """K'_G^T x, entry for entry the transpose of kprime_galerkin."""
        x = _c(x)
        y = np.empty(self.n)
        _load().oracle_kprime_t_galerkin(self.n, self.nq, _p(self.cen), _p(self.nrm), _p(self.area),
                                         _p(self.panels), _p(self.qp), _p(self.qw), _p(x), _p(y))
        return y

    def bt_galerkin(self, v, grad=False):
        """B_G^T v (and its gradient in the charge positions, [nc, 3])."""
        v = _c(v)
        u = np.empty(self.nc)
        h = np.empty((self.nc, 3)) if grad else None
        _load().oracle_bt_galerkin(self.n, self.nq, _p(self.nrm), _p(self.area), _p(self.qp), _p(self.qw),
                                   self.nc, _p(self.xq), _p(v), _p(u),
                                   _p(h) if grad else ctypes.POINTER(ctypes.c_double)())
        return (u, h) if grad else u

    def gradients_galerkin(self, tol: float = 1e-12, restart: int = 30, maxiter: int = 1000):
        """The adjoint gradients of the Galerkin form's energy: as gradients()
        with K' and B replaced by K'_G and B_G (C is the same)."""
        sigma, _ = self.solve_galerkin(tol=tol, restart=restart, maxiter=maxiter)
        lam, _ = self.solve_galerkin(tol=tol, restart=restart, maxiter=maxiter, transpose=True,
                                     b=self.ct(self.q))
        pref = 4.0 * np.pi * KCAL_PER_MOL / (2.0 * self.eps_in)
        phi = self.c(sigma)
        bt, gbt = self.bt_galerkin(lam, grad=True)
        dq = pref * (phi - self.ehat * bt)
        dx = pref * self.q[:, None] * (self.grad_c(sigma) - self.ehat * gbt)
        dg = pref * float(self.q @ phi)
        return dg, dq, dx, sigma, lam

    def kprime_t(self, x):
        x = _c(x)
        y = np.empty(self.n)
        _load().oracle_kprime_t(self.n, self.nq, _p(self.cen), _p(self.nrm), _p(self.qp),
                                _p(self.qw), _p(x), _p(y))
        return y

    def kprime_dense(self):
        K = np.empty((self.n, self.n))
        _load().oracle_kprime_dense(self.n, self.nq, _p(self.cen), _p(self.nrm), _p(self.qp),
                                    _p(self.qw), _p(K))
        return K

    def A(self, x):
        """A x = x + Ehat K' x (Eq. ASC, interior-limit reading)."""
        return _c(x) + self.ehat * self.kprime(x)

    def At(self, x):
        return _c(x) + self.ehat * self.kprime_t(x)

    def bq(self, q=None):
        """Normal field of the charges at the collocation points, E_n = B q."""
        q = self.q if q is None else _c(q)
        E = np.empty(self.n)
        _load().oracle_bq(self.n, _p(self.cen), _p(self.nrm), self.nc, _p(self.xq), _p(q), _p(E))
        return E

    def bq_rows(self, rows, q=None):
        """Rows of B q (the normal field at the collocation points `rows`)."""
        q = self.q if q is None else _c(q)
        rows = np.asarray(rows, dtype=np.int64)
        cen, nrm = _c(self.cen[rows]), _c(self.nrm[rows])
        E = np.empty(rows.shape[0])
        _load().oracle_bq(rows.shape[0], _p(cen), _p(nrm), self.nc, _p(self.xq), _p(q), _p(E))
        return E

    def c_rows(self, s, ks):
        """Entries ks of C s (the potential of the surface charge s at the
        charges ks, Eq. reac)."""
        s = _c(s)
        ks = np.asarray(ks, dtype=np.int64)
        xk = _c(self.xq[ks])
        phi = np.empty(ks.shape[0])
        if self.exact_charge_near:
            _load().oracle_c_exact(self.n, self.nq, _p(self.qp), _p(self.qw), _p(self.cen), _p(self.area),
                                   _p(self.panels), ks.shape[0], _p(xk), _p(s), _p(phi))
        else:
            _load().oracle_c(self.n, self.nq, _p(self.qp), _p(self.qw), ks.shape[0], _p(xk), _p(s), _p(phi))
        return phi

    def bt(self, v):
        v = _c(v)
        u = np.empty(self.nc)
        _load().oracle_bt(self.n, _p(self.cen), _p(self.nrm), self.nc, _p(self.xq), _p(v), _p(u))
        return u

    def c(self, s):
        """phi = C s (Eq. reac with G = 1/(4 pi r))."""
        s = _c(s)
        phi = np.empty(self.nc)
        if self.exact_charge_near:
            _load().oracle_c_exact(self.n, self.nq, _p(self.qp), _p(self.qw), _p(self.cen), _p(self.area),
                                   _p(self.panels), self.nc, _p(self.xq), _p(s), _p(phi))
        else:
            _load().oracle_c(self.n, self.nq, _p(self.qp), _p(self.qw), self.nc, _p(self.xq),
                             _p(s), _p(phi))
        return phi

    def ct(self, u):
        u = _c(u)
        v = np.empty(self.n)
        if self.exact_charge_near:
            _load().oracle_ct_exact(self.n, self.nq, _p(self.qp), _p(self.qw), _p(self.cen), _p(self.area),
                                    _p(self.panels), self.nc, _p(self.xq), _p(u), _p(v))
        else:
            _load().oracle_ct(self.n, self.nq, _p(self.qp), _p(self.qw), self.nc, _p(self.xq),
                              _p(u), _p(v))
        return v

    def grad_c(self, s):
        s = _c(s)
        g = np.empty((self.nc, 3))
        if self.exact_charge_near:
            _load().oracle_grad_c_exact(self.n, self.nq, _p(self.qp), _p(self.qw), _p(self.cen),
                                        _p(self.area), _p(self.panels), self.nc, _p(self.xq), _p(s), _p(g))
        else:
            _load().oracle_grad_c(self.n, self.nq, _p(self.qp), _p(self.qw), self.nc, _p(self.xq),
                                  _p(s), _p(g))
        return g

    def grad_bt(self, v):
        v = _c(v)
        h = np.empty((self.nc, 3))
        _load().oracle_grad_bt(self.n, _p(self.cen), _p(self.nrm), self.nc, _p(self.xq),
                               _p(v), _p(h))
        return h

    # --- solve, energy, BIBEE ----------------------------------------------
    def rhs(self, q=None):
        """b = -Ehat (B q)."""
        return -self.ehat * self.bq(q)

    def solve(self, tol: float = 1e-10, restart: int = 30, maxiter: int = 500, x0=None,
              transpose: bool = False, b=None):
        """sigma from (I + Ehat K') sigma = -Ehat B q by restarted GMRES."""
        op = self.At if transpose else self.A
        b = self.rhs() if b is None else _c(b)
        x, info = gmres(op, b, tol=tol, restart=restart, maxiter=maxiter, x0=x0)
        return x, info

    def energy(self, sigma, q=None):
        """dG [kcal/mol] = 4 pi 332.0637 / (2 eps_in) q . (C sigma)."""
        q = self.q if q is None else _c(q)
        phi = self.c(sigma)
        return 4.0 * np.pi * KCAL_PER_MOL / (2.0 * self.eps_in) * float(q @ phi), phi

    def bibee(self, variant: str = "cfa"):
        lam = BIBEE_LAMBDA[variant]
        sig = bibee_factor(self.eps_in, self.eps_out, lam) * self.bq()
        dg, _ = self.energy(sig)
        return sig, dg

    def gradients(self, tol: float = 1e-12, restart: int = 30, maxiter: int = 1000):
        """d dG / d q [nc] and d dG / d x [nc, 3] by the dense adjoint.

        dG = kappa/(2 eps_in) q^T C A^{-1} (-Ehat) B q, kappa = 4 pi 332.0637.
        lam solves A^T lam = C^T q; then
          d dG/d q_k = kappa/(2 eps_in) [ (C sigma)_k - Ehat (B^T lam)_k ]
          d dG/d x_k = kappa/(2 eps_in) q_k [ grad (C sigma)_k - Ehat sum_i lam_i grad_{x_k} B_ik ].
        """
        sigma, info1 = self.solve(tol=tol, restart=restart, maxiter=maxiter)
        lam, info2 = self.solve(tol=tol, restart=restart, maxiter=maxiter, transpose=True,
                                b=self.ct(self.q))
        pref = 4.0 * np.pi * KCAL_PER_MOL / (2.0 * self.eps_in)
        phi = self.c(sigma)
        dq = pref * (phi - self.ehat * self.bt(lam))
        dx = pref * self.q[:, None] * (self.grad_c(sigma) - self.ehat * self.grad_bt(lam))
        dg = pref * float(self.q @ phi)
        return dg, dq, dx, sigma, lam


def gmres(op, b, tol=1e-10, restart=30, maxiter=500, x0=None):
    """Restarted GMRES(m) (Saad & Schultz 1986): MGS Arnoldi, Givens rotations.

    Returns x and a dict with the iteration count, the recurrence residual and
    the true relative residual |b - op(x)| / |b|.
    """
    b = _c(b)
    n = b.shape[0]
    x = np.zeros(n) if x0 is None else _c(x0).copy()
    bnorm = np.linalg.norm(b)
    if bnorm == 0.0:
        return x, {"iters": 0, "resid": 0.0, "true_resid": 0.0, "converged": True}
    m = int(restart)
    it = 0
    rec = 1.0
    converged = False
    while it < maxiter:
        r = b - op(x)
        beta = np.linalg.norm(r)
        if beta / bnorm <= tol:
            converged = True
            rec = beta / bnorm
            break
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        k = 0
        for j in range(m):
            w = op(V[j])
            it += 1
            for i in range(j + 1):
                H[i, j] = w @ V[i]
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0.0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            k = j + 1
            rec = abs(g[j + 1]) / bnorm
            if rec <= tol or it >= maxiter:
                break
        y = np.zeros(k)
        for i in range(k - 1, -1, -1):
            y[i] = (g[i] - H[i, i + 1:k] @ y[i + 1:k]) / H[i, i]
        x = x + V[:k].T @ y
        if rec <= tol:
            converged = True
            break
    true = np.linalg.norm(b - op(x)) / bnorm
    return x, {"iters": it, "resid": rec, "true_resid": true, "converged": converged}
