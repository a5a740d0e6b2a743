"""Thin ctypes binding of the C ABI declared in ``include/wadg.h``.

Argument marshalling only: every step of the solver runs in the library's
CUDA kernels.  The functions keep the C names; ``Solver`` is a small
convenience wrapper that owns one context.  If the shared library is missing
the import fails loudly (there is no fallback implementation).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
# WADG_LIB selects another build of the library (the checked diagnostic
# build, _lib/libwadg_checked.so) for the whole process
LIB_PATH = os.environ.get("WADG_LIB") or os.path.join(HERE, "_lib", "libwadg.so")

WADG_OK, WADG_EINVAL, WADG_ENOMEM, WADG_ECUDA, WADG_ESTATE = 0, 1, 2, 3, 4
WADG_ENOTFOUND, WADG_ETIMEOUT, WADG_ENONFINITE, WADG_EUNSUPPORTED = 5, 6, 7, 8
STATUS_NAMES = {0: "OK", 1: "EINVAL", 2: "ENOMEM", 3: "ECUDA", 4: "ESTATE",
                5: "ENOTFOUND", 6: "ETIMEOUT", 7: "ENONFINITE", 8: "EUNSUPPORTED"}
PRECISION = {"fp64": 0, "fp32": 1, "tf32": 2, "bf16": 3}
SCHEME = {"waa": 0, "stored": 1, "ec": 2}


class WadgError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class wadg_pml_profile(C.Structure):
    _fields_ = [("u0", C.c_double * 3), ("L", C.c_double * 3),
                ("sigma_max", C.c_double * 3), ("p_sigma", C.c_double * 3),
                ("kappa_max", C.c_double * 3), ("eps0", C.c_double)]


class wadg_dipole(C.Structure):
    _fields_ = [("x", C.c_double * 3), ("dir", C.c_double * 3), ("t0", C.c_double),
                ("width", C.c_double), ("amplitude", C.c_double), ("batch", C.c_int32)]


_P = C.c_void_p
_D = C.POINTER(C.c_double)
_I64 = C.POINTER(C.c_int64)
_SIG = {
    "wadg_create": [C.c_int, C.c_int, C.c_int32, C.c_int, _P, C.POINTER(_P)],
    "wadg_destroy": [_P],
    "wadg_set_mesh": [_P, C.c_int64, _D, C.c_int64, _I64],
    "wadg_set_mesh_periodic": [_P, C.c_int64, _D, C.c_int64, _I64, _I64],
    "wadg_set_materials": [_P, _D, _D],
    "wadg_set_pml_profile": [_P, C.POINTER(wadg_pml_profile), C.c_int],
    "wadg_set_sources": [_P, C.c_int32, C.POINTER(wadg_dipole)],
    "wadg_set_probes": [_P, C.c_int32, _D],
    "wadg_set_quadrature": [_P, C.c_int32, _D],
    "wadg_set_state": [_P, _P, C.c_double, C.c_int],
    "wadg_get_state": [_P, _P, _D, C.c_int],
    "wadg_state_bytes": [_P, C.POINTER(C.c_size_t)],
    "wadg_bind_state": [_P, _P, C.c_size_t],
    "wadg_transfer_bytes": [_P, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)],
    "wadg_rk_stage": [_P, C.c_int, C.c_double, C.c_double],
    "wadg_run_steps": [_P, C.c_int64, C.c_double, _D],
    "wadg_run_steps_noalloc": [_P, C.c_int64, C.c_double, _D],
    "wadg_stable_dt": [_P, C.c_double, _D],
    "wadg_profile_stage": [_P, C.c_int, C.c_double, _D],
    "wadg_adjoint": [_P, C.c_int64, C.c_double, C.c_int32, _D, _D, _D, _D],
    "wadg_objective": [_P, _D],
    "wadg_memory_report": [_P, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t),
                           C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)],
    "wadg_mesh_info": [_P, _I64, _I64, C.POINTER(C.c_int32), C.POINTER(C.c_int32)],
    "wadg_synchronize": [_P],
    "wadg_arm_wait_timeout": [_P],
    "wadg_set_memory_limit": [_P, C.c_size_t, _P],
    "wadg_reference_operator": [C.c_int, C.c_int, _D, C.c_int64, _I64],
    "wadg_fma_peak": [C.c_int, C.c_int, _D],
    "wadg_group_create": [C.c_int32, C.POINTER(_P), C.POINTER(_P)],
    "wadg_group_destroy": [_P],
    "wadg_group_autotune": [_P, _D, C.c_int32, _D],
    "wadg_group_info": [_P] + [C.POINTER(C.c_int32)] * 10,
    "wadg_group_set_tuning": [_P, C.c_int32, C.c_int32, C.c_int32, C.c_int32, C.c_int32],
    "wadg_group_run_steps": [_P, C.c_int64, _D, C.POINTER(_D)],
}

_lib = None


def load(path: str = LIB_PATH):
    """Load the shared library (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"libwadg.so not built at {path}; run "
                          "paper_2006_02551_gb300.build.build()")
    lib = C.CDLL(path)
    for name, args in _SIG.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = C.c_int
    lib.wadg_last_error.argtypes = [_P]
    lib.wadg_last_error.restype = C.c_char_p
    lib.wadg_group_last_error.argtypes = [_P]
    lib.wadg_group_last_error.restype = C.c_char_p
    _lib = lib
    return lib


def exported_symbols():
    return list(_SIG) + ["wadg_last_error", "wadg_group_last_error"]


def _ptr(a):
    return a.ctypes.data_as(_D) if a is not None else None


def _check(st, ctx=None):
    if st != WADG_OK:
        msg = load().wadg_last_error(ctx)
        raise WadgError(st, (msg or b"").decode())


def reference_operator(N: int, which: int) -> np.ndarray:
    lib = load()
    n = C.c_int64(0)
    _check(lib.wadg_reference_operator(N, which, None, 0, C.byref(n)))
    out = np.empty(n.value)
    _check(lib.wadg_reference_operator(N, which, _ptr(out), n.value, C.byref(n)))
    return out


def fma_peak(device=0, fp64=False) -> float:
    """Measured CUDA-core FMA throughput (TFLOP/s) of a device."""
    lib = load()
    t = C.c_double()
    _check(lib.wadg_fma_peak(device, 1 if fp64 else 0, C.byref(t)))
    return t.value


def make_profile(u0, L, sigma_max, p_sigma, kappa_max=1.0, eps0=1.0):
    p = wadg_pml_profile()
    for name, v in (("u0", u0), ("L", L), ("sigma_max", sigma_max),
                    ("p_sigma", p_sigma), ("kappa_max", kappa_max)):
        arr = getattr(p, name)
        vals = v if np.ndim(v) else (v, v, v)
        for i in range(3):
            arr[i] = float(vals[i])
    p.eps0 = eps0
    return p


class Solver:
    """One library context (one device, one stream)."""

    def __init__(self, N, precision="fp64", n_batch=1, device=0, stream=None):
        lib = load()
        self.lib = lib
        self.N, self.n_batch, self.precision = N, n_batch, precision
        ctx = _P()
        _check(lib.wadg_create(N, PRECISION[precision], n_batch, device,
                               _P(stream) if stream else None, C.byref(ctx)))
        self.ctx = ctx

    def close(self):
        if self.ctx:
            self.lib.wadg_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _c(self, st):
        _check(st, self.ctx)

    def set_mesh(self, vxyz, etov, vcanon=None):
        """vcanon: optional periodic vertex representatives (wadg_set_mesh_periodic)."""
        v = np.ascontiguousarray(vxyz, dtype=np.float64)
        e = np.ascontiguousarray(etov, dtype=np.int64)
        if vcanon is None:
            self._c(self.lib.wadg_set_mesh(self.ctx, v.shape[0], _ptr(v), e.shape[0],
                                           e.ctypes.data_as(_I64)))
        else:
            c = np.ascontiguousarray(vcanon, dtype=np.int64)
            self._c(self.lib.wadg_set_mesh_periodic(self.ctx, v.shape[0], _ptr(v), e.shape[0],
                                                    e.ctypes.data_as(_I64),
                                                    c.ctypes.data_as(_I64)))
        self.K = e.shape[0]

    def set_materials(self, eps_r=None, mu_r=None):
        er = None if eps_r is None else np.ascontiguousarray(eps_r, np.float64)
        mr = None if mu_r is None else np.ascontiguousarray(mu_r, np.float64)
        self._c(self.lib.wadg_set_materials(self.ctx, _ptr(er), _ptr(mr)))

    def set_pml(self, profile, scheme="waa"):
        if profile is None:
            self._c(self.lib.wadg_set_pml_profile(self.ctx, None, SCHEME[scheme]))
            return
        if not isinstance(profile, wadg_pml_profile):
            profile = make_profile(profile.u0, profile.L, profile.sigma_max,
                                   profile.p_sigma, profile.kappa_max, profile.eps0)
        self._c(self.lib.wadg_set_pml_profile(self.ctx, C.byref(profile), SCHEME[scheme]))

    def set_sources(self, dipoles):
        arr = (wadg_dipole * max(1, len(dipoles)))()
        for i, d in enumerate(dipoles):
            for k in range(3):
                arr[i].x[k] = d.x[k]
                arr[i].dir[k] = d.dir[k]
            arr[i].t0, arr[i].width, arr[i].amplitude = d.t0, d.width, d.amplitude
            arr[i].batch = d.batch
        self._c(self.lib.wadg_set_sources(self.ctx, len(dipoles), arr))

    def set_quadrature(self, rstw=None):
        """Volume quadrature of the PML terms: rows (r, s, t, w) on the
        reference tetrahedron, or None for the default (N+1)^3-point rule."""
        if rstw is None:
            self._c(self.lib.wadg_set_quadrature(self.ctx, 0, None))
            return
        a = np.ascontiguousarray(np.asarray(rstw, np.float64).reshape(-1, 4))
        self._c(self.lib.wadg_set_quadrature(self.ctx, a.shape[0], _ptr(a)))

    def set_probes(self, xyz):
        p = np.ascontiguousarray(np.asarray(xyz, np.float64).reshape(-1, 3))
        self.n_probe = p.shape[0]
        self._c(self.lib.wadg_set_probes(self.ctx, p.shape[0], _ptr(p)))

    def info(self):
        K, K1 = C.c_int64(), C.c_int64()
        Np, Nq = C.c_int32(), C.c_int32()
        self._c(self.lib.wadg_mesh_info(self.ctx, C.byref(K), C.byref(K1), C.byref(Np),
                                        C.byref(Nq)))
        return dict(K=K.value, K_pml=K1.value, Np=Np.value, Nq=Nq.value)

    def state_shape(self):
        """Shape of the state array of set_state / get_state: [n_batch][K][12][Np]
        (E, H, P^E, P^H per element in the caller's element order)."""
        inf = self.info()
        return (self.n_batch, inf["K"], 12, inf["Np"])

    _state_shape = state_shape

    def _device_ptr(self, x):
        """Address of a contiguous float64 device tensor of the state's shape
        (any object with data_ptr(), is_cuda, dtype and shape, e.g. torch)."""
        if tuple(x.shape) != self._state_shape() or str(x.dtype) != "torch.float64" \
                or not x.is_cuda or not x.is_contiguous():
            raise ValueError(f"device state must be a contiguous float64 CUDA tensor of shape "
                             f"{self._state_shape()}")
        return _P(x.data_ptr())

    def set_state(self, q=None, t=0.0):
        """q: host array (numpy) or a CUDA tensor (device exchange, no host
        copy; ordered on the context's stream) of shape [nb][K][12][Np]."""
        if q is not None and hasattr(q, "data_ptr") and getattr(q, "is_cuda", False):
            self._c(self.lib.wadg_set_state(self.ctx, self._device_ptr(q), t, 1))
            return
        a = None if q is None else np.ascontiguousarray(q, np.float64)
        self._c(self.lib.wadg_set_state(self.ctx, _P(a.ctypes.data) if a is not None else None,
                                        t, 0))

    def get_state(self, out=None):
        """(q, t).  With out = a CUDA tensor of the state's shape the state is
        written there on the device (no host copy) and out is returned."""
        t = C.c_double()
        if out is not None:
            self._c(self.lib.wadg_get_state(self.ctx, self._device_ptr(out), C.byref(t), 1))
            return out, t.value
        q = np.empty(self._state_shape())
        self._c(self.lib.wadg_get_state(self.ctx, _P(q.ctypes.data), C.byref(t), 0))
        return q, t.value

    def state_bytes(self):
        n = C.c_size_t()
        self._c(self.lib.wadg_state_bytes(self.ctx, C.byref(n)))
        return n.value

    def bind_state(self, buf):
        """Keep the state buffers in caller-owned device memory buf (a CUDA
        tensor of at least state_bytes() bytes, 256-byte aligned), or
        None to return them to the library.  The solver keeps a reference to
        buf while it is bound."""
        if buf is None:
            self._c(self.lib.wadg_bind_state(self.ctx, None, 0))
            self._bound = None
            return
        nbytes = buf.numel() * buf.element_size()
        self._c(self.lib.wadg_bind_state(self.ctx, _P(buf.data_ptr()), nbytes))
        self._bound = buf

    def transfer_bytes(self):
        """(host-to-device, device-to-host) bytes copied by this context."""
        a, b = C.c_size_t(), C.c_size_t()
        self._c(self.lib.wadg_transfer_bytes(self.ctx, C.byref(a), C.byref(b)))
        return a.value, b.value

    def rk_stage(self, stage, t, dt):
        self._c(self.lib.wadg_rk_stage(self.ctx, stage, t, dt))

    def run_steps(self, nsteps, dt, record=True):
        out = None
        if record and getattr(self, "n_probe", 0):
            out = np.empty((nsteps, self.n_probe, 6, self.n_batch))
        self._c(self.lib.wadg_run_steps(self.ctx, nsteps, dt, _ptr(out)))
        return out

    def profile_stage(self, reps, dt):
        ms = np.zeros(2)
        self._c(self.lib.wadg_profile_stage(self.ctx, reps, dt, _ptr(ms)))
        return ms

    def adjoint(self, nsteps, dt, ckpt_every=45):
        """(J [nb], dJ/deps_r [nb][K], dJ/dsigma_max [nb][3], dJ/dp_sigma [nb][3])."""
        nb = self.n_batch
        J = np.empty(nb)
        ge = np.empty((nb, self.info()["K"]))
        gs = np.empty((nb, 3))
        gp = np.empty((nb, 3))
        self._c(self.lib.wadg_adjoint(self.ctx, nsteps, dt, ckpt_every, _ptr(J), _ptr(ge),
                                      _ptr(gs), _ptr(gp)))
        return J, ge, gs, gp

    def run_steps_noalloc(self, nsteps, dt, record=True):
        """run_steps through the entry point that allocates no device memory."""
        out = None
        if record and getattr(self, "n_probe", 0):
            out = np.empty((nsteps, self.n_probe, 6, self.n_batch))
        self._c(self.lib.wadg_run_steps_noalloc(self.ctx, nsteps, dt, _ptr(out)))
        return out

    def stable_dt(self, cfl=1.0):
        d = C.c_double()
        self._c(self.lib.wadg_stable_dt(self.ctx, cfl, C.byref(d)))
        return d.value

    def objective(self):
        J = np.empty(self.n_batch)
        self._c(self.lib.wadg_objective(self.ctx, _ptr(J)))
        return J

    def memory_report(self):
        v = [C.c_size_t() for _ in range(4)]
        self._c(self.lib.wadg_memory_report(self.ctx, *[C.byref(x) for x in v]))
        return dict(state=v[0].value, pml_coeff=v[1].value, operators=v[2].value,
                    geometry=v[3].value)

    def synchronize(self):
        self._c(self.lib.wadg_synchronize(self.ctx))

    def set_memory_limit(self, nbytes):
        """Cap the device bytes this context may hold (0: no cap); returns
        the bytes it holds now.  Allocations past the cap raise
        WadgError(ENOMEM) and leave the context usable."""
        held = C.c_size_t()
        self._c(self.lib.wadg_set_memory_limit(self.ctx, nbytes, C.byref(held)))
        return held.value

    def arm_wait_timeout(self):
        """Failure-detection test aid (TF32/BF16 contexts): the next
        tensor-core stage launch withholds one product signal, its bounded
        wait runs out and the stepping call raises WadgError(ETIMEOUT)."""
        self._c(self.lib.wadg_arm_wait_timeout(self.ctx))


class Group:
    """Several solvers advanced together (wadg_group_*): per stage one grouped
    launch per (order, element class) variant (FP32 CUDA-core members), or
    every member's own kernels (any precision), in turn or on parallel graph
    branches.  Refers to the solvers: close it before them."""

    def __init__(self, solvers):
        self.lib = load()
        self.solvers = list(solvers)
        self.g = None
        arr = (_P * len(self.solvers))(*[s.ctx for s in self.solvers])
        g = _P()
        st = self.lib.wadg_group_create(len(self.solvers), arr, C.byref(g))
        if st != WADG_OK:
            raise WadgError(st, (self.lib.wadg_group_last_error(None) or b"").decode())
        self.g = g

    def _c(self, st):
        if st != WADG_OK:
            msg = self.lib.wadg_group_last_error(self.g)
            raise WadgError(st, (msg or b"").decode())

    def close(self):
        if self.g:
            self.lib.wadg_group_destroy(self.g)
            self.g = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def autotune(self, dts, reps=20):
        d = np.ascontiguousarray(dts, np.float64)
        ms = C.c_double()
        self._c(self.lib.wadg_group_autotune(self.g, _ptr(d), reps, C.byref(ms)))
        return ms.value

    def set_tuning(self, per_item=False, parallel=True, share=False, tile_divisor=1,
                   blocks_per_sm=1):
        """Fix the launch shape without timing (see autotune)."""
        self._c(self.lib.wadg_group_set_tuning(self.g, int(per_item), int(parallel), int(share),
                                               tile_divisor, blocks_per_sm))

    def info(self):
        v = [C.c_int32() for _ in range(10)]
        self._c(self.lib.wadg_group_info(self.g, *[C.byref(x) for x in v]))
        return dict(blocks=v[0].value, threads=v[1].value, blocks_per_sm=v[2].value,
                    tile_divisor=v[3].value, items=v[4].value, variants=v[5].value,
                    parallel=bool(v[6].value), share=bool(v[7].value), clusters=v[8].value,
                    per_item=bool(v[9].value))

    def run_steps(self, nsteps, dts, record=True):
        d = np.ascontiguousarray(dts, np.float64)
        outs = []
        ptrs = (_D * len(self.solvers))()
        for i, s in enumerate(self.solvers):
            o = None
            if record and getattr(s, "n_probe", 0):
                o = np.empty((nsteps, s.n_probe, 6, s.n_batch))
                ptrs[i] = _ptr(o)
            outs.append(o)
        self._c(self.lib.wadg_group_run_steps(self.g, nsteps, _ptr(d), ptrs))
        return outs
