"""Python binding of libbem, the GB300 FMM-BEM solver (arXiv:1007.4591).

The functions below have the names of the C entry points declared in
``include/bem.h`` and only marshal arguments: every step of the computation
runs in the CUDA library.  Arrays may be torch CUDA tensors (device pointers,
used in place) or numpy / CPU arrays (host pointers, staged by the library).
There is no CPU fallback: importing this package without the built
``lib/libbem.so`` raises.

A small convenience class, :class:`Mesh`, owns a handle and exposes the same
operations with array allocation done here (plumbing only).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libbem.so")

BEM_OK = 0
BEM_EINVAL = -1
BEM_ENOMEM = -2
BEM_ECUDA = -3
BEM_ENOCONV = -4
BEM_ETIMEOUT = -5
BEM_EUNSUPPORTED = -6

BEM_MIXED = 0
BEM_FP64 = 1
BEM_NEAR_QUADRATURE = 1
BEM_NEAR_EXACT = 2
BEM_BIBEE_CFA = 0
BEM_BIBEE_P = 1
BEM_BIBEE_PLUS_HALF = 2
BEM_FLAG_NO_FAR = 1
BEM_FLAG_NO_NEAR = 2
BEM_FLAG_NO_NEARTAB = 4
BEM_FLAG_CHECK_CHARGES = 8
BEM_FLAG_M2L_REDUCE = 16
BEM_FLAG_CHARGE_NEAR_EXACT = 32
BEM_FLAG_P2M_FROM_POINTS = 64
BEM_CHARGE_AUTO = 0
BEM_CHARGE_FMM = 1
BEM_CHARGE_DIRECT = 2
BEM_M2L_AUTO = 0
BEM_M2L_DENSE = 1
BEM_M2L_DIRECT = 2
BEM_M2L_TC = 3
BEM_NOALLOC_SCRATCH_FLOATS = 1 << 21  # the allocation-free entry point's largest n_t

ERROR_NAMES = {0: "BEM_OK", -1: "BEM_EINVAL", -2: "BEM_ENOMEM", -3: "BEM_ECUDA",
               -4: "BEM_ENOCONV", -5: "BEM_ETIMEOUT", -6: "BEM_EUNSUPPORTED"}


class bem_options(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("p", ctypes.c_int), ("leaf_size", ctypes.c_int),
                ("depth", ctypes.c_int), ("quad_points", ctypes.c_int),
                ("gmres_restart", ctypes.c_int), ("max_iter", ctypes.c_int),
                ("tol", ctypes.c_double), ("flags", ctypes.c_uint), ("near_table", ctypes.c_int),
                ("charge_mode", ctypes.c_int), ("m2l_mode", ctypes.c_int), ("graph", ctypes.c_int),
                ("galerkin", ctypes.c_int)]


class bem_solve_stats(ctypes.Structure):
    _fields_ = [("iterations", ctypes.c_int), ("restarts", ctypes.c_int),
                ("converged", ctypes.c_int), ("resid", ctypes.c_double),
                ("true_resid", ctypes.c_double), ("ms_rhs", ctypes.c_double),
                ("ms_gmres", ctypes.c_double), ("ms_total", ctypes.c_double)]


class bem_mesh_info(ctypes.Structure):
    _fields_ = [("n_p", ctypes.c_int64), ("n_c", ctypes.c_int64), ("depth", ctypes.c_int),
                ("p", ctypes.c_int), ("precision", ctypes.c_int), ("leaves", ctypes.c_int64),
                ("cells", ctypes.c_int64), ("p2p_pairs", ctypes.c_int64),
                ("m2l_pairs", ctypes.c_int64), ("m2m_pairs", ctypes.c_int64),
                ("source_points", ctypes.c_int64), ("near_table_nnz", ctypes.c_int64),
                ("root_side", ctypes.c_double), ("device_bytes", ctypes.c_size_t),
                ("ms_build", ctypes.c_double), ("p2m_segments", ctypes.c_int64)]


_vp = ctypes.c_void_p
_SIGS = {
    "bem_options_default": [ctypes.POINTER(bem_options)],
    "bem_mesh_create": [_vp, ctypes.c_int64, _vp, ctypes.c_int64, ctypes.c_double,
                        ctypes.c_double, ctypes.POINTER(bem_options), _vp, ctypes.POINTER(_vp)],
    "bem_mesh_destroy": [_vp],
    "bem_set_charges": [_vp, _vp, ctypes.c_int64],
    "bem_matvec": [_vp, _vp, _vp],
    "bem_matvec_t": [_vp, _vp, _vp],
    "bem_rhs": [_vp, _vp],
    "bem_solve": [_vp, _vp, _vp, ctypes.POINTER(bem_solve_stats)],
    "bem_bibee": [_vp, ctypes.c_int, _vp, _vp],
    "bem_energy": [_vp, _vp, _vp, _vp],
    "bem_energy_backward": [_vp, ctypes.c_double, _vp, _vp],
    "bem_mesh_info_get": [_vp, ctypes.POINTER(bem_mesh_info)],
    "bem_set_profiling": [_vp, ctypes.c_int],
    "bem_set_wait_budget": [_vp, ctypes.c_longlong],
    "bem_set_device_memory_cap": [ctypes.c_size_t],
    "bem_last_phase_ms": [_vp, _vp],
    "bem_last_m2l_ms": [_vp, _vp],
    "bem_last_near_ms": [_vp, _vp],
    "bem_fp32_peak": [_vp],
    "bem_last_error": [],
    "bem_batch_solve": [_vp, ctypes.c_int, ctypes.c_int, _vp, _vp, _vp, _vp, _vp],
    "bem_normal_field_noalloc": [_vp, _vp, ctypes.c_int64, _vp, ctypes.c_int64, _vp, _vp],
    "bem_autotune": [_vp, ctypes.c_int64, _vp, ctypes.c_int64, ctypes.c_double, ctypes.c_double,
                     ctypes.c_double, ctypes.POINTER(bem_options)],
}

_lib = None


def load_library(path: str | None = None):
    """Load libbem.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"libbem.so not found at {path}: build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    lib = ctypes.CDLL(path)
    for name, args in _SIGS.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_char_p if name == "bem_last_error" else ctypes.c_int
    _lib = lib
    return lib


class BemError(RuntimeError):
    def __init__(self, code: int, where: str):
        self.code = code
        msg = load_library().bem_last_error().decode(errors="replace")
        super().__init__(f"{where}: {ERROR_NAMES.get(code, code)}: {msg}")


def _check(code: int, where: str, allow=()):
    if code != BEM_OK and code not in allow:
        raise BemError(code, where)
    return code


def _ptr(a):
    """Raw pointer of a torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(a.data_ptr())
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(a.ctypes.data)
    raise TypeError(f"unsupported array type {type(a)}")


def _check_f64(a, n, name):
    if a is None:
        return
    dt = getattr(a, "dtype", None)
    ok = str(dt) in ("float64", "torch.float64")
    if not ok:
        raise TypeError(f"{name} must be float64")
    cnt = a.numel() if hasattr(a, "numel") else a.size
    if cnt != n:
        raise ValueError(f"{name} must have {n} elements")


# ---------------------------------------------------------------- C-ABI names
def bem_options_default() -> bem_options:
    o = bem_options()
    _check(load_library().bem_options_default(ctypes.byref(o)), "bem_options_default")
    return o


def bem_mesh_create(panels, charges, eps_in, eps_out, opt: bem_options | None = None,
                    stream=None):
    lib = load_library()
    n_p = int(panels.shape[0])
    n_c = int(charges.shape[0]) if charges is not None else 0
    _check_f64(panels, n_p * 9, "panels")
    if charges is not None:
        _check_f64(charges, n_c * 4, "charges")
    h = ctypes.c_void_p()
    o = opt if opt is not None else bem_options_default()
    st = ctypes.c_void_p(stream) if stream is not None else None
    _check(lib.bem_mesh_create(_ptr(panels), n_p, _ptr(charges), n_c, float(eps_in),
                               float(eps_out), ctypes.byref(o), st, ctypes.byref(h)),
           "bem_mesh_create")
    return h


def bem_mesh_destroy(h):
    return _check(load_library().bem_mesh_destroy(h), "bem_mesh_destroy")


def bem_set_charges(h, charges):
    n_c = int(charges.shape[0])
    return _check(load_library().bem_set_charges(h, _ptr(charges), n_c), "bem_set_charges")


def bem_matvec(h, x, y):
    return _check(load_library().bem_matvec(h, _ptr(x), _ptr(y)), "bem_matvec")


def bem_matvec_t(h, x, y):
    return _check(load_library().bem_matvec_t(h, _ptr(x), _ptr(y)), "bem_matvec_t")


def bem_rhs(h, b):
    return _check(load_library().bem_rhs(h, _ptr(b)), "bem_rhs")


def bem_solve(h, x0, sigma, allow_noconv: bool = False):
    st = bem_solve_stats()
    allow = (BEM_ENOCONV,) if allow_noconv else ()
    rc = _check(load_library().bem_solve(h, _ptr(x0), _ptr(sigma), ctypes.byref(st)),
                "bem_solve", allow)
    return rc, st


def bem_bibee(h, variant: int, sigma_hat=None) -> float:
    dg = ctypes.c_double()
    _check(load_library().bem_bibee(h, int(variant), _ptr(sigma_hat), ctypes.byref(dg)),
           "bem_bibee")
    return dg.value


def bem_energy(h, sigma, phi=None) -> float:
    dg = ctypes.c_double()
    _check(load_library().bem_energy(h, _ptr(sigma), ctypes.byref(dg), _ptr(phi)), "bem_energy")
    return dg.value


def bem_energy_backward(h, grad_out: float, dq=None, dx=None):
    return _check(load_library().bem_energy_backward(h, float(grad_out), _ptr(dq), _ptr(dx)),
                  "bem_energy_backward")


def bem_mesh_info_get(h) -> bem_mesh_info:
    info = bem_mesh_info()
    _check(load_library().bem_mesh_info_get(h, ctypes.byref(info)), "bem_mesh_info_get")
    return info


def bem_set_profiling(h, enable: bool):
    return _check(load_library().bem_set_profiling(h, 1 if enable else 0), "bem_set_profiling")


def bem_set_wait_budget(h, cycles: int):
    return _check(load_library().bem_set_wait_budget(h, int(cycles)), "bem_set_wait_budget")


def bem_set_device_memory_cap(nbytes: int):
    return _check(load_library().bem_set_device_memory_cap(int(nbytes)), "bem_set_device_memory_cap")


def bem_last_phase_ms(h):
    t = np.zeros(7)
    _check(load_library().bem_last_phase_ms(h, _ptr(t)), "bem_last_phase_ms")
    return dict(zip(["p2m", "m2m", "m2l", "l2l", "l2p", "p2p", "epilogue"], t.tolist()))


def bem_last_m2l_ms(h):
    t = np.zeros(3)
    _check(load_library().bem_last_m2l_ms(h, _ptr(t)), "bem_last_m2l_ms")
    return dict(zip(["split", "tc"], t.tolist()[:2]))


def bem_fp32_peak() -> float:
    """Measured FP32 throughput of the current device, TFLOP/s."""
    t = ctypes.c_double()
    _check(load_library().bem_fp32_peak(ctypes.byref(t)), "bem_fp32_peak")
    return float(t.value)


def bem_last_near_ms(h):
    t = np.zeros(2)
    _check(load_library().bem_last_near_ms(h, _ptr(t)), "bem_last_near_ms")
    return dict(zip(["strength", "p2p"], t.tolist()))


def bem_batch_solve(meshes, threads: int = 8, sigmas=None):
    """Solve every mesh of `meshes` (Mesh objects or raw handles) concurrently.

    Returns (dG, dG_cfa, dG_p, stats) as numpy arrays / list of dicts.
    `sigmas` (optional) is a list of f64 arrays receiving each solution."""
    n = len(meshes)
    hs = (ctypes.c_void_p * n)(*[m.h if hasattr(m, "h") else m for m in meshes])
    dg = np.zeros(n)
    dc = np.zeros(n)
    dp = np.zeros(n)
    st = (bem_solve_stats * n)()
    sp = None
    if sigmas is not None:
        sp = (ctypes.c_void_p * n)(*[_ptr(s) for s in sigmas])
    rc = load_library().bem_batch_solve(hs, n, int(threads), sp, _ptr(dg), _ptr(dc), _ptr(dp),
                                        ctypes.cast(st, ctypes.c_void_p))
    _check(rc, "bem_batch_solve", (BEM_ENOCONV,))
    stats = [{f: getattr(s, f) for f, _ in s._fields_} for s in st]
    return dg, dc, dp, stats


def bem_autotune(panels, charges, eps_in, eps_out, target: float = 1e-5,
                 opt: bem_options | None = None) -> bem_options:
    o = opt if opt is not None else bem_options_default()
    n_p = int(panels.shape[0])
    n_c = int(charges.shape[0]) if charges is not None else 0
    _check(load_library().bem_autotune(_ptr(panels), n_p, _ptr(charges), n_c, float(eps_in),
                                       float(eps_out), float(target), ctypes.byref(o)),
           "bem_autotune")
    return o


def bem_normal_field_noalloc(targets, normals, charges, field, stream=None):
    """Normal field of point charges at points, allocating nothing on the GPU
    (for callers that cannot allocate; device tensors only, see include/bem.h).
    Queued on `stream` (a raw cudaStream_t, None = legacy default)."""
    n_t = int(targets.shape[0])
    n_c = int(charges.shape[0])
    for a, name in ((targets, "targets"), (normals, "normals"), (charges, "charges"), (field, "field")):
        if not getattr(a, "is_cuda", False):
            raise TypeError(f"{name} must be a CUDA tensor (this entry point takes device memory only)")
    _check_f64(targets, 3 * n_t, "targets")
    _check_f64(normals, 3 * n_t, "normals")
    _check_f64(charges, 4 * n_c, "charges")
    _check_f64(field, n_t, "field")
    st = ctypes.c_void_p(stream) if stream is not None else None
    return _check(load_library().bem_normal_field_noalloc(_ptr(targets), _ptr(normals), n_t,
                                                          _ptr(charges), n_c, _ptr(field), st),
                  "bem_normal_field_noalloc")


def bem_last_error() -> str:
    return load_library().bem_last_error().decode(errors="replace")


# --------------------------------------------------------------- convenience
def make_options(**kw) -> bem_options:
    o = bem_options_default()
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


class Mesh:
    """Owns one bem_mesh handle; arrays are torch CUDA tensors (f64)."""

    def __init__(self, panels, charges, eps_in, eps_out, stream=None, **opts):
        import torch
        self.torch = torch
        self.device = torch.device("cuda", torch.cuda.current_device())
        pan = torch.as_tensor(panels, dtype=torch.float64).reshape(-1, 3, 3).contiguous()
        ch = torch.as_tensor(charges, dtype=torch.float64).reshape(-1, 4).contiguous()
        self.n_p, self.n_c = int(pan.shape[0]), int(ch.shape[0])
        self.opt = make_options(**opts)
        self.stream = stream if stream is not None else torch.cuda.current_stream().cuda_stream
        self.h = bem_mesh_create(pan.to(self.device), ch.to(self.device), eps_in, eps_out,
                                 self.opt, self.stream)

    def close(self):
        if getattr(self, "h", None) is not None:
            bem_mesh_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _vec(self, n):
        return self.torch.empty(n, dtype=self.torch.float64, device=self.device)

    def _dev(self, x, n):
        t = self.torch.as_tensor(x, dtype=self.torch.float64).to(self.device).contiguous()
        if t.numel() != n:
            raise ValueError(f"expected {n} values")
        return t

    def info(self) -> dict:
        i = bem_mesh_info_get(self.h)
        return {f: getattr(i, f) for f, _ in i._fields_}

    def matvec(self, x):
        y = self._vec(self.n_p)
        bem_matvec(self.h, self._dev(x, self.n_p), y)
        return y

    def matvec_t(self, x):
        y = self._vec(self.n_p)
        bem_matvec_t(self.h, self._dev(x, self.n_p), y)
        return y

    def rhs(self):
        b = self._vec(self.n_p)
        bem_rhs(self.h, b)
        return b

    def solve(self, x0=None, allow_noconv=False):
        s = self._vec(self.n_p)
        rc, st = bem_solve(self.h, None if x0 is None else self._dev(x0, self.n_p), s,
                           allow_noconv)
        return s, {f: getattr(st, f) for f, _ in st._fields_}

    def energy(self, sigma, want_phi=False):
        phi = self._vec(self.n_c) if want_phi else None
        dg = bem_energy(self.h, self._dev(sigma, self.n_p), phi)
        return (dg, phi) if want_phi else dg

    def bibee(self, variant=BEM_BIBEE_CFA, want_sigma=False):
        s = self._vec(self.n_p) if want_sigma else None
        dg = bem_bibee(self.h, variant, s)
        return (dg, s) if want_sigma else dg

    def energy_backward(self, grad_out=1.0):
        dq = self._vec(self.n_c)
        dx = self._vec(self.n_c * 3)
        bem_energy_backward(self.h, grad_out, dq, dx)
        return dq, dx.reshape(self.n_c, 3)

    def set_charges(self, charges):
        ch = self.torch.as_tensor(charges, dtype=self.torch.float64).reshape(-1, 4).contiguous()
        bem_set_charges(self.h, ch.to(self.device))
        self.n_c = int(ch.shape[0])


# ------------------------------------------------------------------ autograd
def _energy_function():
    import torch

    class SolvationEnergy(torch.autograd.Function):
        """dG(charges) with the adjoint gradient (bem_energy_backward).

        charges: [n_c, 4] float64 tensor (x, y, z, q).  Forward: the charge
        tree is rebuilt for the new charges (the panel tree and near-field
        tables are the mesh's), the BEM system is solved and dG returned in
        kcal/mol.  Backward: one transposed solve, then d dG/dq and d dG/dx.
        """

        @staticmethod
        def forward(ctx, charges, mesh):
            mesh.set_charges(charges.detach().to(torch.float64).contiguous())
            sig, st = mesh.solve()
            dg = mesh.energy(sig)
            ctx.mesh = mesh
            return charges.new_tensor(dg)

        @staticmethod
        def backward(ctx, g):
            dq, dx = ctx.mesh.energy_backward(float(g))
            grad = torch.cat([dx, dq[:, None]], dim=1)
            return grad, None

    return SolvationEnergy


_SE = None


def solvation_energy(mesh: "Mesh", charges):
    """Differentiable electrostatic solvation energy (kcal/mol) of `charges`."""
    global _SE
    if _SE is None:
        _SE = _energy_function()
    return _SE.apply(charges, mesh)

def autotune_cached(panels, charges, eps_in, eps_out, target: float = 1e-5, cache: str | None = None):
    """bem_autotune with its choice kept in a JSON file: the (leaf_size, p)
    found for these exact panels, charges, dielectrics and target are read
    back instead of re-tuned.  Returns a dict {"leaf_size", "p", "cached"}."""
    import hashlib
    import json
    pan = np.ascontiguousarray(panels, dtype=np.float64)
    ch = np.ascontiguousarray(charges, dtype=np.float64)
    h = hashlib.sha256()
    for a in (pan, ch, np.array([eps_in, eps_out, target], dtype=np.float64)):
        h.update(a.tobytes())
    key = h.hexdigest()
    table = {}
    if cache and os.path.exists(cache):
        with open(cache) as f:
            table = json.load(f)
        if key in table:
            return dict(table[key], cached=True)
    o = bem_autotune(pan, ch, eps_in, eps_out, target=target)
    entry = {"leaf_size": int(o.leaf_size), "p": int(o.p)}
    if cache:
        table[key] = entry
        tmp = cache + ".tmp"
        with open(tmp, "w") as f:
            json.dump(table, f, indent=1)
        os.replace(tmp, cache)
    return dict(entry, cached=False)


# ------------------------------------------------------------ workflows
def binding_free_energy(complex_, receptor, ligand, threads: int = 3, **opts):
    """Electrostatic binding free energy (Eq. binding, Sec. 5):
        dG_bind = dG_complex - dG_receptor - dG_ligand,
    each term a full solve on its own mesh; the three solves run as one
    bem_batch_solve.  Arguments are molecules with .panels, .charges,
    .eps_in, .eps_out (e.g. synth.complex_pair()); opts go to make_options.
    Returns (dG_bind, (dG_complex, dG_receptor, dG_ligand)) in kcal/mol."""
    meshes = [Mesh(m.panels, m.charges, m.eps_in, m.eps_out, **opts) for m in (complex_, receptor, ligand)]
    try:
        dg, _, _, _ = bem_batch_solve(meshes, threads=threads)
    finally:
        for g in meshes:
            g.close()
    return float(dg[0] - dg[1] - dg[2]), (float(dg[0]), float(dg[1]), float(dg[2]))


def superposition_energy(isolated, system, copies: int, **opts):
    """The crowded-solution heuristic (Sec. 5): the induced surface charge of
    one isolated molecule is reused on every copy in the system instead of
    solving the whole system self-consistently.  `system`'s panels must be
    `copies` rigid copies of `isolated`'s panels, copy after copy (rigid
    motions leave the per-panel induced charge unchanged), with the copies'
    charges.  Returns a dict with
        dG_coupled     energy of the self-consistent solve of the system,
        dG_superposed  energy of the system with the isolated induced charge
                       on every copy (interactions between copies included),
        dG_isolated    copies x the isolated molecule's energy,
    all in kcal/mol."""
    with Mesh(isolated.panels, isolated.charges, isolated.eps_in, isolated.eps_out, **opts) as g:
        s_iso, _ = g.solve()
        e_iso = g.energy(s_iso)
    with Mesh(system.panels, system.charges, system.eps_in, system.eps_out, **opts) as G:
        if G.n_p != copies * int(s_iso.shape[0]):
            raise ValueError("system panels are not `copies` copies of the isolated molecule")
        e_sup = G.energy(s_iso.repeat(copies))
        s, _ = G.solve()
        e = G.energy(s)
    return {"dG_coupled": float(e), "dG_superposed": float(e_sup), "dG_isolated": float(copies * e_iso)}

