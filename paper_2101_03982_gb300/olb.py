"""Thin ctypes binding of ``libolb.so`` (C ABI in ``include/olb.h``).

Argument marshalling only: every step of the method runs in the library's
CUDA kernels.  Device arrays are torch CUDA tensors (passed by data pointer on
the simulation's stream); host arrays are numpy arrays.  There is no CPU
fallback: if the library is missing, the first call raises.
"""
import ctypes
import os

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
_LIBPATH = os.path.join(_PKG, "libolb.so")

VELOCITY_SETS = {"D2Q9": 0, "D2Q19": 1, "D2Q25": 2, "D3Q13": 3, "D3Q21": 4, "D3Q27": 5, "D3V27": 6, "D3Q45": 7}
STORAGES = {"fp64": 0, "fp32": 1, "bf16": 2, "fp16": 3}
ERRORS = {0: "OLB_OK", -1: "OLB_EINVAL", -2: "OLB_ENOMEM", -3: "OLB_ECUDA", -4: "OLB_ENONFINITE",
          -5: "OLB_ETIMEOUT", -6: "OLB_EBOUNDS", -7: "OLB_EUNSUPPORTED", -8: "OLB_ESTATE"}


class OlbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int), ("n", ctypes.c_int * 3), ("dx", ctypes.c_double)]


class Options(ctypes.Structure):
    _fields_ = [("interp_order", ctypes.c_int), ("storage", ctypes.c_int), ("cs_scale", ctypes.c_double),
                ("compressible", ctypes.c_int), ("gamma", ctypes.c_double), ("mu", ctypes.c_double),
                ("mu_exponent", ctypes.c_double), ("prandtl", ctypes.c_double), ("rho0", ctypes.c_double), ("allow_inexact", ctypes.c_int), ("log_every", ctypes.c_int),
                ("kernel", ctypes.c_int), ("stream", ctypes.c_void_p)]


_lib = None


def lib():
    """The loaded library (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIBPATH):
            raise RuntimeError(f"{_LIBPATH} is missing: build it with `python -m paper_2101_03982_gb300.build`")
        L = ctypes.CDLL(_LIBPATH)
        vp, i, d, sz = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
        dp, ip = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)
        sig = {
            "olb_default_options": (None, [ctypes.POINTER(Options)]),
            "olb_velocity_set_info": (i, [i, ip, ip, dp, dp, ip]),
            "olb_velocity_set_table": (i, [i, vp, vp]),
            "olb_create": (i, [ctypes.POINTER(Grid), i, i, d, d, ctypes.POINTER(Options), ctypes.POINTER(vp)]),
            "olb_destroy": (i, [vp]),
            "olb_shape": (i, [vp, ip, ip, ctypes.POINTER(sz), ip, ip]),
            "olb_stencil": (i, [vp, vp, vp]),
            "olb_init_fields": (i, [vp, vp, vp, vp, i]),
            "olb_step": (i, [vp, i]),
            "olb_moments": (i, [vp, vp, vp, vp, i]),
            "olb_reductions": (i, [vp, vp]),
            "olb_kinetic_energy": (i, [vp, dp, dp]),
            "olb_get_populations": (i, [vp, vp, i]),
            "olb_set_populations": (i, [vp, vp, i]),
            "olb_state_bytes": (sz, [vp]),
            "olb_get_state": (i, [vp, vp, sz, i]),
            "olb_set_state": (i, [vp, vp, sz, i]),
            "olb_synchronize": (i, [vp, i]),
            "olb_set_wait_polls": (i, [vp, ctypes.c_longlong]),
            "olb_set_interpolation": (i, [vp, i]),
            "olb_state_sums_noalloc": (i, [i, ctypes.POINTER(Grid), i, d, d, vp, vp, vp]),
            "olb_enstrophy": (i, [vp, dp]),
            "olb_tape_reserve": (i, [vp, i]),
            "olb_tape_record": (i, [vp, i]),
            "olb_tape_adjoint": (i, [vp, vp, i, i]),
            "olb_adjoint_step": (i, [vp, vp, vp, i]),
            "olb_moments_vjp": (i, [vp, vp, vp, vp, i]),
            "olb_equilibrium_vjp": (i, [vp, vp, vp, vp, vp, vp, i]),
            "olb_fp64_fma_peak": (i, [vp, dp]),
            "olb_set_x_boundary": (i, [vp, i, d, dp, d]),
            "olb_glc_stencil": (i, [i, d, ip, dp]),
            "olb_strerror": (ctypes.c_char_p, [i]),
            "olb_last_error": (ctypes.c_char_p, []),
        }
        for name, (res, args) in sig.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(rc):
    if rc != 0:
        raise OlbError(rc, lib().olb_last_error().decode())
    return rc


def velocity_set_info(name):
    """(Q, D, c_s, max |xi_alpha|, degree) of a velocity set, unscaled."""
    Q, D, deg = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    cs, mx = ctypes.c_double(), ctypes.c_double()
    _check(lib().olb_velocity_set_info(VELOCITY_SETS[name], ctypes.byref(Q), ctypes.byref(D), ctypes.byref(cs),
                                       ctypes.byref(mx), ctypes.byref(deg)))
    return Q.value, D.value, cs.value, mx.value, deg.value


def fp64_fma_peak(stream=None):
    """Measured FP64 FMA throughput of the current device in flop/s."""
    out = ctypes.c_double()
    _check(lib().olb_fp64_fma_peak(stream, ctypes.byref(out)))
    return out.value


def glc_stencil(p, shift):
    """Per-residue (first (p,), W (p, p+1)) of the cell-wise GLC interpolation."""
    first = np.zeros(p, dtype=np.int32)
    W = np.zeros((p, p + 1))
    _check(lib().olb_glc_stencil(int(p), float(shift), first.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                 W.ctypes.data_as(ctypes.POINTER(ctypes.c_double))))
    return first, W


def velocity_set_table(name):
    """Abscissae (Q, D) and weights (Q,) of a velocity set as the library holds them."""
    Q, D, _, _, _ = velocity_set_info(name)
    xi = np.zeros((Q, D))
    w = np.zeros(Q)
    _check(lib().olb_velocity_set_table(VELOCITY_SETS[name], xi.ctypes.data, w.ctypes.data))
    return xi, w


def _ptr(a):
    """(pointer, on_device) of a torch tensor or numpy array (contiguous FP64 or raw)."""
    if a is None:
        return None, 0
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), 1 if a.is_cuda else 0
    if not a.flags["C_CONTIGUOUS"]:
        raise ValueError("array must be C-contiguous")
    return a.ctypes.data, 0


class Sim:
    """One simulation: a handle of the C library.

    shape is (nx, ny) or (nx, ny, nz); arrays use the [z][y][x] memory order,
    so a field has numpy/torch shape (ny, nx) or (nz, ny, nx).
    """

    def __init__(self, shape, dx, velocity_set, hermite_order, tau, dt, interp_order=3, storage="fp64",
                 cs_scale=1.0, compressible=False, gamma=1.4, mu=0.0, rho0=1.0, allow_inexact=False,
                 log_every=1, kernel="auto", stream=None, mu_exponent=0.0, prandtl=1.0):
        L = lib()
        g = Grid()
        g.dim = len(shape)
        n = list(shape) + [1] * (3 - len(shape))
        for k in range(3):
            g.n[k] = int(n[k])
        g.dx = float(dx)
        o = Options()
        L.olb_default_options(ctypes.byref(o))
        o.interp_order = int(interp_order)
        o.storage = STORAGES[storage]
        o.cs_scale = float(cs_scale)
        o.compressible = int(bool(compressible))
        o.gamma = float(gamma)
        o.mu = float(mu)
        o.mu_exponent = float(mu_exponent)
        o.prandtl = float(prandtl)
        o.rho0 = float(rho0)
        o.allow_inexact = int(bool(allow_inexact))
        o.log_every = int(log_every)
        o.kernel = {"auto": 0, "generic": 1, "twophase": 2}[kernel]
        if stream is None:
            try:
                import torch
                if torch.cuda.is_available():
                    stream = torch.cuda.current_stream().cuda_stream
            except ImportError:
                stream = None
        o.stream = stream
        self._h = ctypes.c_void_p()
        _check(L.olb_create(ctypes.byref(g), VELOCITY_SETS[velocity_set], int(hermite_order), float(tau),
                            float(dt), ctypes.byref(o), ctypes.byref(self._h)))
        self.shape = tuple(int(s) for s in shape)
        self.grid_shape = tuple(reversed(self.shape))  # array shape (z, y, x)
        Q, planes, nodes, dim, eb = (ctypes.c_int(), ctypes.c_int(), ctypes.c_size_t(), ctypes.c_int(),
                                     ctypes.c_int())
        _check(L.olb_shape(self._h, ctypes.byref(Q), ctypes.byref(planes), ctypes.byref(nodes), ctypes.byref(dim),
                           ctypes.byref(eb)))
        self.Q, self.planes, self.nodes, self.dim, self.elem_bytes = Q.value, planes.value, nodes.value, dim.value, eb.value
        self.interp_order = int(interp_order)
        self.storage = storage
        self.stream = stream

    # -- lifetime ----------------------------------------------------------
    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            _check(lib().olb_destroy(self._h))
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- calls -------------------------------------------------------------
    def init_fields(self, rho, u, theta=None):
        pr, dr = _ptr(rho)
        pu, du = _ptr(u)
        pt, dt = _ptr(theta)
        if dr != du or (theta is not None and dt != dr):
            raise ValueError("fields must all be on the device or all on the host")
        _check(lib().olb_init_fields(self._h, pr, pu, pt, dr))

    def step(self, n=1):
        _check(lib().olb_step(self._h, int(n)))

    def moments(self, rho, u, theta=None):
        """Write rho (n), u (D, n) and theta (n) of the stored state into the given arrays."""
        pr, dr = _ptr(rho)
        pu, _ = _ptr(u)
        pt, _ = _ptr(theta)
        _check(lib().olb_moments(self._h, pr, pu, pt, dr))

    def reductions(self, check=True):
        out = np.zeros(8)
        rc = lib().olb_reductions(self._h, out.ctypes.data)
        if check and rc != 0:
            _check(rc)
        return dict(k=out[0], k_rho=out[1], eps=out[2], mass=out[3], momentum=out[4:4 + self.dim].copy(),
                    nonfinite=int(out[7]), rc=rc)

    def kinetic_energy(self):
        k, e = ctypes.c_double(), ctypes.c_double()
        _check(lib().olb_kinetic_energy(self._h, ctypes.byref(k), ctypes.byref(e)))
        return k.value, e.value

    def enstrophy(self):
        """Mean |curl u|^2 of the current state (fourth-order central differences)."""
        e = ctypes.c_double()
        _check(lib().olb_enstrophy(self._h, ctypes.byref(e)))
        return e.value

    def get_populations(self, out):
        p, d = _ptr(out)
        _check(lib().olb_get_populations(self._h, p, d))
        return out

    def set_populations(self, f):
        p, d = _ptr(f)
        _check(lib().olb_set_populations(self._h, p, d))

    def state_bytes(self):
        return int(lib().olb_state_bytes(self._h))

    def get_state(self, buf, nbytes=None):
        p, d = _ptr(buf)
        _check(lib().olb_get_state(self._h, p, nbytes or self.state_bytes(), d))
        return buf

    def set_state(self, buf, nbytes=None):
        p, d = _ptr(buf)
        _check(lib().olb_set_state(self._h, p, nbytes or self.state_bytes(), d))

    def stencil(self):
        """(m0 (Q, 3), W (Q, 3, p+1)) of the pull as the library built it."""
        m0 = np.zeros((self.Q, 3), dtype=np.int32)
        W = np.zeros((self.Q, 3, self.interp_order + 1))
        _check(lib().olb_stencil(self._h, m0.ctypes.data, W.ctypes.data))
        return m0, W

    def set_x_boundary(self, kind, rho=1.0, u=None, theta=1.0):
        """kind "periodic", or "inflow_outflow" with the inflow state (rho, u (D,), theta)."""
        k = {"periodic": 0, "inflow_outflow": 1}[kind]
        uu = np.zeros(3) if u is None else np.ascontiguousarray(np.asarray(u, dtype=np.float64))
        _check(lib().olb_set_x_boundary(self._h, k, float(rho), uu.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                        float(theta)))

    def synchronize(self, timeout_ms=0):
        _check(lib().olb_synchronize(self._h, int(timeout_ms)))

    def set_interpolation(self, scheme):
        """"uniform" (equidistant Lagrange stencil) or "glc" (the paper's cell-wise GLC interpolation)."""
        _check(lib().olb_set_interpolation(self._h, {"uniform": 0, "glc": 1}[scheme]))

    def set_wait_polls(self, polls):
        """Bound of the step kernels' staging waits (< 0: the default; 0: give up at once)."""
        _check(lib().olb_set_wait_polls(self._h, int(polls)))

    # -- adjoint of the isothermal step ----------------------------------------
    @property
    def adjoint_dtype(self):
        """Element type of adjoint arrays: 'float64' for FP64 storage, 'float32' for FP32."""
        return "float64" if self.storage == "fp64" else "float32"

    def tape_reserve(self, nslots):
        _check(lib().olb_tape_reserve(self._h, int(nslots)))

    def tape_record(self, n):
        _check(lib().olb_tape_record(self._h, int(n)))

    def tape_adjoint(self, lam, n):
        """lam (Q, *grid) in: dJ/d(state after the last recorded step); out: n steps earlier."""
        p, d = _ptr(lam)
        _check(lib().olb_tape_adjoint(self._h, p, int(n), d))
        return lam

    def adjoint_step(self, fwd_state, lam):
        ps, ds = _ptr(fwd_state)
        pl, dl = _ptr(lam)
        if ds != dl:
            raise ValueError("state and adjoint must both be on the device or both on the host")
        _check(lib().olb_adjoint_step(self._h, ps, pl, dl))
        return lam

    def moments_vjp(self, grad_rho, grad_u, lam):
        pr, dr = _ptr(grad_rho)
        pu, du = _ptr(grad_u)
        pl, dl = _ptr(lam)
        for a, d in ((grad_rho, dr), (grad_u, du)):
            if a is not None and d != dl:
                raise ValueError("gradients and adjoint must all be on the device or all on the host")
        _check(lib().olb_moments_vjp(self._h, pr, pu, pl, dl))
        return lam

    def equilibrium_vjp(self, rho, u, lam, grad_rho, grad_u):
        ptrs = [_ptr(a) for a in (rho, u, lam, grad_rho, grad_u)]
        if len({d for _, d in ptrs}) != 1:
            raise ValueError("arrays must all be on the device or all on the host")
        _check(lib().olb_equilibrium_vjp(self._h, *[p for p, _ in ptrs], ptrs[0][1]))
        return grad_rho, grad_u
