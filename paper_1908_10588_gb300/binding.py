"""Thin ctypes binding of libvibtdvp (include/vibtdvp.h).

Argument marshalling only: every step of the 2TDVP path runs in the
library's CUDA kernels. The library is built in-tree by `build.py`; if it is
missing this module raises instead of falling back to anything else.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libvibtdvp.so")

VB_OK, VB_EINVAL, VB_ENOMEM, VB_ECUDA, VB_ENOCONV, VB_ETIMEOUT, VB_ESTATE = 0, -1, -2, -3, -4, -5, -6
VB_FP64, VB_MIXED = 0, 1
_NAMES = {0: "VB_OK", -1: "VB_EINVAL", -2: "VB_ENOMEM", -3: "VB_ECUDA", -4: "VB_ENOCONV",
          -5: "VB_ETIMEOUT", -6: "VB_ESTATE"}

EXPORTED = [
    "vb_last_error", "vb_version", "mpo_build", "mpo_destroy", "mpo_n_sites", "mpo_site_dims",
    "mpo_site_tensor", "mps_create", "mps_create_from_tensors", "mps_destroy", "mps_n_sites",
    "mps_bond_dims", "mps_get_site", "tdvp2_sweep", "measure_populations", "vb_heff2_apply",
    "vb_heff1_apply", "vb_heff_work_elems", "vb_env_left_update", "vb_env_right_update",
    "vb_env_work_elems", "vb_herm_eig_top", "vb_eig_work_bytes", "vb_kernel_launches",
    "vb_profile_enable", "vb_profile_read", "vb_herm_eig_top_noalloc", "mps_overlap", "mps_energy",
    "tdvp2_sweep_batched", "tdvp1_sweep", "vb_site_order_cost", "vb_site_order_search", "vb_site_order_rule",
    "mps_get_tensor", "vb_test_raise_wait_flag", "vb_spectrum", "tdvp2_population_gradient",
    "global_krylov_step", "vb_autotune",
]


class VbError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{_NAMES.get(code, code)}: {msg}")
        self.code = code


class vb_model(C.Structure):
    _fields_ = [("n_el", C.c_int), ("e0", C.POINTER(C.c_double)), ("v0", C.POINTER(C.c_double)),
                ("n_modes", C.c_int), ("omega", C.POINTER(C.c_double)), ("levels", C.POINTER(C.c_int)),
                ("g1", C.POINTER(C.c_double)), ("n_g2", C.c_int), ("g2_idx", C.POINTER(C.c_int)),
                ("g2_val", C.POINTER(C.c_double)), ("site_order", C.POINTER(C.c_int)),
                ("include_zpe", C.c_int)]


class vb_allocator(C.Structure):
    _fields_ = [("alloc", C.c_void_p), ("free", C.c_void_p), ("ctx", C.c_void_p)]


class vb_mps_opts(C.Structure):
    _fields_ = [("m_cap", C.c_int), ("dtype", C.c_int), ("pad_full", C.c_int), ("krylov_cap", C.c_int),
                ("cuda_stream", C.c_void_p), ("alloc", C.POINTER(vb_allocator))]


class vb_tdvp_opts(C.Structure):
    _fields_ = [("m_max", C.c_int), ("eps", C.c_double), ("zero_floor", C.c_double),
                ("krylov_max", C.c_int), ("krylov_tol", C.c_double), ("on_noconv", C.c_int)]


class vb_profile(C.Structure):
    _fields_ = [("ms", C.c_double * 24), ("calls", C.c_longlong * 24), ("heff_flops", C.c_double * 2),
                ("krylov_flops", C.c_double), ("flops", C.c_double * 24), ("bytes", C.c_double * 24)]


PHASES = ["heff2", "heff1", "krylov", "split", "env", "merge", "split_rho", "split_eigval", "split_eigvec",
          "split_out", "split_subspace_products", "split_subspace_orth", "eigvec_invit", "eigvec_gram_schmidt",
          "eigvec_backtransform", "split_rayleigh_ritz", "split_ritz_fp32", "split_ritz_fp64",
          "split_orth_cholesky", "split_orth_products", "heff_tc_legs", "heff_sparse_legs", "heff_prep",
          "ritz_jacobi"]  # ritz_jacobi: its "flops" entry counts Jacobi sweeps


class vb_order_opts(C.Structure):
    _fields_ = [("m_max", C.c_int), ("w_flops", C.c_double), ("w_size", C.c_double), ("w_coupling", C.c_double),
                ("iters", C.c_int), ("seed", C.c_ulonglong), ("n_strong", C.c_int)]


class vb_order_cost(C.Structure):
    _fields_ = [("heff_flops", C.c_double), ("tensor_elems", C.c_double), ("max_tensor", C.c_double),
                ("coupling_dist", C.c_double), ("objective", C.c_double), ("max_w", C.c_int)]


class vb_krylov_info(C.Structure):
    _fields_ = [("r", C.c_int), ("converged", C.c_int), ("disc_basis", C.c_double), ("disc_final", C.c_double),
                ("max_bond_basis", C.c_int)]


class vb_sweep_stats(C.Structure):
    _fields_ = [("max_bond", C.c_int), ("discarded_weight", C.c_double), ("krylov_iters_max", C.c_int),
                ("krylov_iters_total", C.c_int), ("noconv", C.c_int)]


_lib = None


def lib():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_1908_10588_gb300.build.build()")
    L = C.CDLL(LIB_PATH)
    vp, i, d, sz = C.c_void_p, C.c_int, C.c_double, C.c_size_t
    sig = {
        "vb_last_error": (C.c_char_p, []),
        "vb_version": (i, []),
        "mpo_build": (i, [C.POINTER(vb_model), C.POINTER(vp)]),
        "mpo_destroy": (i, [vp]),
        "mpo_n_sites": (i, [vp]),
        "mpo_site_dims": (i, [vp, i, C.POINTER(i), C.POINTER(i), C.POINTER(i)]),
        "mpo_site_tensor": (i, [vp, i, vp]),
        "mps_create": (i, [vp, C.POINTER(i), C.POINTER(vb_mps_opts), C.POINTER(vp)]),
        "mps_create_from_tensors": (i, [vp, C.POINTER(i), C.POINTER(vp), C.POINTER(vb_mps_opts), C.POINTER(vp)]),
        "mps_destroy": (i, [vp]),
        "mps_n_sites": (i, [vp]),
        "mps_bond_dims": (i, [vp, C.POINTER(i)]),
        "mps_get_site": (i, [vp, i, vp]),
        "mps_get_tensor": (i, [vp, i, vp, vp]),
        "vb_test_raise_wait_flag": (i, [vp]),
        "vb_spectrum": (i, [vp, i, d, d, vp, i, vp, vp]),
        "tdvp2_population_gradient": (i, [vp, vp, d, i, C.POINTER(vb_tdvp_opts), i, i, vp, vp, vp, i, vp, vp]),
        "global_krylov_step": (i, [vp, vp, d, C.POINTER(vb_tdvp_opts), i, d, C.POINTER(vb_krylov_info)]),
        "vb_autotune": (i, [i, i, C.POINTER(i), C.c_char_p, i]),
        "tdvp2_sweep": (i, [vp, vp, d, C.POINTER(vb_tdvp_opts), C.POINTER(vb_sweep_stats)]),
        "measure_populations": (i, [vp, vp]),
        "tdvp1_sweep": (i, [vp, vp, d, C.POINTER(vb_tdvp_opts), C.POINTER(vb_sweep_stats)]),
        "mps_overlap": (i, [vp, vp, vp]),
        "mps_energy": (i, [vp, vp]),
        "tdvp2_sweep_batched": (i, [C.POINTER(vp), C.POINTER(vp), i, d, C.POINTER(vb_tdvp_opts),
                                    C.POINTER(vb_sweep_stats)]),
        "vb_heff2_apply": (i, [vp, i, i, i, vp, vp, vp, vp, vp, i, vp]),
        "vb_heff1_apply": (i, [vp, i, i, i, vp, vp, vp, vp, vp, i, vp]),
        "vb_heff_work_elems": (sz, [vp, i, i, i, i]),
        "vb_env_left_update": (i, [vp, i, i, i, vp, vp, vp, vp, vp]),
        "vb_env_right_update": (i, [vp, i, i, i, vp, vp, vp, vp, vp]),
        "vb_env_work_elems": (sz, [vp, i, i, i]),
        "vb_herm_eig_top": (i, [i, vp, i, i, vp, vp, vp, vp]),
        "vb_eig_work_bytes": (sz, [i, i]),
        "vb_herm_eig_top_noalloc": (i, [i, vp, i, i, vp, vp, vp]),
        "vb_kernel_launches": (C.c_ulonglong, []),
        "vb_profile_enable": (i, [i]),
        "vb_profile_read": (i, [C.POINTER(vb_profile), i]),
        "vb_site_order_cost": (i, [C.POINTER(vb_model), vp, C.POINTER(vb_order_opts), C.POINTER(vb_order_cost),
                                   vp, vp]),
        "vb_site_order_search": (i, [C.POINTER(vb_model), C.POINTER(vb_order_opts), vp, C.POINTER(vb_order_cost)]),
        "vb_site_order_rule": (i, [C.POINTER(vb_model), i, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    _lib = L
    return L


def check(code):
    if code != VB_OK:
        msg = lib().vb_last_error()
        raise VbError(code, msg.decode() if msg else "")


def _dp(a: np.ndarray, ctype):
    return a.ctypes.data_as(C.POINTER(ctype))


def _ptr(x):
    """Device or host address of a torch tensor / numpy array / int."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if hasattr(x, "data_ptr"):
        return x.data_ptr()
    return x.ctypes.data


def _stream_ptr(stream):
    if stream is None:
        return None
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream



def _model_struct(model: dict, keep: list) -> "vb_model":
    """vb_model view of a model dict (see vibmodels); the arrays it points to
    are appended to `keep`, which must outlive the struct."""
    def arr(a, dt):
        a = np.ascontiguousarray(a, dtype=dt)
        keep.append(a)
        return a

    e0 = arr(model["e0"], np.float64)
    v0 = arr(model["v0"], np.float64).reshape(-1)
    lev = arr(model["levels"], np.int32)
    g1 = arr(model["g1"], np.float64).reshape(-1)
    g2 = model["g2"]
    g2i = arr(np.array([[I, J, i, j] for (I, J, i, j, _) in g2], dtype=np.int32).reshape(-1, 4), np.int32)
    g2v = arr(np.array([v for (*_, v) in g2], dtype=np.float64), np.float64)
    om = arr(model["omega"], np.float64)
    so = model.get("site_order")
    m = vb_model()
    m.n_el = int(model["n_el"])
    m.e0 = _dp(e0, C.c_double)
    m.v0 = _dp(v0, C.c_double)
    m.n_modes = om.size
    m.omega = _dp(om, C.c_double)
    m.levels = _dp(lev, C.c_int)
    m.g1 = _dp(g1, C.c_double)
    m.n_g2 = len(g2)
    m.g2_idx = _dp(g2i, C.c_int) if len(g2) else None
    m.g2_val = _dp(g2v, C.c_double) if len(g2) else None
    m.site_order = _dp(arr(so, np.int32), C.c_int) if so is not None else None
    m.include_zpe = int(model.get("include_zpe", 1))
    return m


# ----------------------------------------------------------------- MPO
class Mpo:
    """MPO of a vibronic model dict (see vibmodels); owns the C handle."""

    def __init__(self, model: dict):
        L = lib()
        self._keep = []
        m = _model_struct(model, self._keep)
        self.n_el = int(model["n_el"])
        h = C.c_void_p()
        check(L.mpo_build(C.byref(m), C.byref(h)))
        self.h = h
        self._keep = []

    @property
    def n_sites(self) -> int:
        return lib().mpo_n_sites(self.h)

    def site_dims(self, p: int):
        a, b, c = C.c_int(), C.c_int(), C.c_int()
        check(lib().mpo_site_dims(self.h, p, C.byref(a), C.byref(b), C.byref(c)))
        return a.value, b.value, c.value

    def site_tensor(self, p: int) -> np.ndarray:
        wl, d, wr = self.site_dims(p)
        out = np.zeros((wl, d, d, wr))
        check(lib().mpo_site_tensor(self.h, p, out.ctypes.data))
        return out

    def close(self):
        if self.h:
            lib().mpo_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------- MPS
class Mps:
    """MPS handle (center on site 0) with its device buffers."""

    def __init__(self, mpo: Mpo, init_index=None, m_cap: int = 64, dtype: int = VB_FP64,
                 pad_full: bool = False, krylov_cap: int = 40, stream=None, tensors=None):
        L = lib()
        self.mpo = mpo
        o = vb_mps_opts()
        o.m_cap = m_cap
        o.dtype = dtype
        o.pad_full = int(pad_full)
        o.krylov_cap = krylov_cap
        o.cuda_stream = _stream_ptr(stream)
        o.alloc = None
        h = C.c_void_p()
        if tensors is None:
            idx = (C.c_int * mpo.n_sites)(*[int(x) for x in init_index])
            check(L.mps_create(mpo.h, idx, C.byref(o), C.byref(h)))
        else:
            ts = [np.ascontiguousarray(t, dtype=np.complex128) for t in tensors]
            bonds = (C.c_int * max(1, len(ts) - 1))(*[t.shape[2] for t in ts[:-1]])
            ptrs = (C.c_void_p * len(ts))(*[t.ctypes.data for t in ts])
            check(L.mps_create_from_tensors(mpo.h, bonds, ptrs, C.byref(o), C.byref(h)))
        self.h = h

    @property
    def n_sites(self) -> int:
        return lib().mps_n_sites(self.h)

    def bond_dims(self):
        n = self.n_sites
        out = (C.c_int * max(1, n - 1))()
        check(lib().mps_bond_dims(self.h, out))
        return list(out)[: n - 1]

    def site(self, p: int) -> np.ndarray:
        dims = [self.mpo.site_dims(q)[1] for q in range(self.n_sites)]
        b = [1] + self.bond_dims() + [1]
        out = np.zeros((b[p], dims[p], b[p + 1]), dtype=np.complex128)
        check(lib().mps_get_site(self.h, p, out.ctypes.data))
        return out

    def tensors(self):
        return [self.site(p) for p in range(self.n_sites)]

    def site_shape(self, p: int):
        b = [1] + self.bond_dims() + [1]
        return (b[p], self.mpo.site_dims(p)[1], b[p + 1])

    def get_tensor(self, p: int, out, stream=None):
        """Copy site p device to device into `out` (a caller-owned device
        buffer, e.g. a complex128 torch tensor of `site_shape(p)`), mps_get_tensor."""
        check(lib().mps_get_tensor(self.h, p, _ptr(out), _stream_ptr(stream)))
        return out

    def raise_wait_flag(self):
        """Test hook: set the device flag a timed-out tensor-core wait raises
        (vb_test_raise_wait_flag); the next sweep returns VB_ETIMEOUT."""
        check(lib().vb_test_raise_wait_flag(self.h))

    def sweep(self, dt_fs: float, m_max: int, eps: float = 0.0, zero_floor: float = 1e-14,
              krylov_max: int = 30, krylov_tol: float = 1e-13, on_noconv: int = 0):
        o = vb_tdvp_opts(m_max, eps, zero_floor, krylov_max, krylov_tol, on_noconv)
        st = vb_sweep_stats()
        check(lib().tdvp2_sweep(self.h, self.mpo.h, float(dt_fs), C.byref(o), C.byref(st)))
        return st

    def sweep1(self, dt_fs: float, krylov_max: int = 30, krylov_tol: float = 1e-13, on_noconv: int = 0):
        """One one-site TDVP step at the current bond dimensions (tdvp1_sweep)."""
        o = vb_tdvp_opts(1, 0.0, 0.0, krylov_max, krylov_tol, on_noconv)
        st = vb_sweep_stats()
        check(lib().tdvp1_sweep(self.h, self.mpo.h, float(dt_fs), C.byref(o), C.byref(st)))
        return st

    def population_gradient(self, dt_fs: float, n_steps: int, params, el_state: int, m_max: int,
                            eps: float = 0.0, zero_floor: float = 1e-14, krylov_max: int = 30,
                            krylov_tol: float = 1e-13, checkpoint_every: int = 10):
        """Propagate n_steps 2TDVP steps and return (populations at t,
        dP_el_state/dg for params [(mode, i, j), ...]) (tdvp2_population_gradient)."""
        o = vb_tdvp_opts(m_max, eps, zero_floor, krylov_max, krylov_tol, 0)
        pm = np.ascontiguousarray([p[0] for p in params], dtype=np.int32)
        pi = np.ascontiguousarray([p[1] for p in params], dtype=np.int32)
        pj = np.ascontiguousarray([p[2] for p in params], dtype=np.int32)
        pops = np.zeros(self.mpo.n_el)
        grad = np.zeros(max(1, len(params)))
        check(lib().tdvp2_population_gradient(self.h, self.mpo.h, float(dt_fs), int(n_steps), C.byref(o),
                                              int(el_state), len(params), pm.ctypes.data, pi.ctypes.data,
                                              pj.ctypes.data, int(checkpoint_every), pops.ctypes.data,
                                              grad.ctypes.data))
        return pops, grad[: len(params)]

    def global_krylov(self, dt_fs: float, m_max: int, eps: float = 0.0, zero_floor: float = 1e-14,
                      r_max: int = 20, tol: float = 1e-12):
        """One global Krylov step (global_krylov_step); returns its info."""
        o = vb_tdvp_opts(m_max, eps, zero_floor, 30, 1e-13, 0)
        inf = vb_krylov_info()
        check(lib().global_krylov_step(self.h, self.mpo.h, float(dt_fs), C.byref(o), int(r_max), float(tol),
                                       C.byref(inf)))
        return inf

    def populations(self) -> np.ndarray:
        out = np.zeros(self.mpo.n_el)
        check(lib().measure_populations(self.h, out.ctypes.data))
        return out

    def overlap(self, other: "Mps") -> complex:
        """<self|other> (mps_overlap); with self the initial state this is C(t)."""
        out = np.zeros(2)
        check(lib().mps_overlap(self.h, other.h, out.ctypes.data))
        return complex(out[0], out[1])

    def energy(self) -> float:
        """<psi|H|psi> / <psi|psi> in eV (mps_energy)."""
        out = np.zeros(1)
        check(lib().mps_energy(self.h, out.ctypes.data))
        return float(out[0])

    def save(self, path: str):
        """Checkpoint: bond dimensions and site tensors (host copies) to an .npz
        file; `Mps.load` recreates the handle from it."""
        ts = self.tensors()
        np.savez(path, n_sites=len(ts), **{f"site{p}": t for p, t in enumerate(ts)})

    @classmethod
    def load(cls, mpo: Mpo, path: str, **kw) -> "Mps":
        """Handle from a checkpoint written by `save` (same MPO; options as for
        the constructor: m_cap, dtype, krylov_cap, stream)."""
        with np.load(path) as z:
            ts = [z[f"site{p}"] for p in range(int(z["n_sites"]))]
        return cls(mpo, tensors=ts, **kw)

    def close(self):
        if self.h:
            lib().mps_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sweep_batched(states, dt_fs: float, m_max: int, eps: float = 0.0, zero_floor: float = 1e-14,
                  krylov_max: int = 30, krylov_tol: float = 1e-13, on_noconv: int = 0):
    """One 2TDVP step for each state (tdvp2_sweep_batched); states created on
    different streams run concurrently. Returns the per-state statistics."""
    n = len(states)
    hs = (C.c_void_p * max(1, n))(*[s.h for s in states])
    ms = (C.c_void_p * max(1, n))(*[s.mpo.h for s in states])
    o = vb_tdvp_opts(m_max, eps, zero_floor, krylov_max, krylov_tol, on_noconv)
    st = (vb_sweep_stats * max(1, n))()
    check(lib().tdvp2_sweep_batched(hs, ms, n, float(dt_fs), C.byref(o), st))
    return [st[i] for i in range(n)]


# ------------------------------------------- single operations (device ptrs)
def vb_heff_work_elems(mpo: Mpo, site: int, mL: int, mR: int, two_site: bool) -> int:
    return int(lib().vb_heff_work_elems(mpo.h, site, mL, mR, int(two_site)))


def vb_heff2_apply(mpo: Mpo, i, mL, mR, L, R, theta, y, work, dtype=VB_FP64, stream=None):
    check(lib().vb_heff2_apply(mpo.h, i, mL, mR, _ptr(L), _ptr(R), _ptr(theta), _ptr(y), _ptr(work),
                               dtype, _stream_ptr(stream)))


def vb_heff1_apply(mpo: Mpo, j, mL, mR, L, R, Cc, y, work, dtype=VB_FP64, stream=None):
    check(lib().vb_heff1_apply(mpo.h, j, mL, mR, _ptr(L), _ptr(R), _ptr(Cc), _ptr(y), _ptr(work),
                               dtype, _stream_ptr(stream)))


def vb_env_work_elems(mpo: Mpo, site, mL, mR) -> int:
    return int(lib().vb_env_work_elems(mpo.h, site, mL, mR))


def vb_env_left_update(mpo: Mpo, p, mL, mR, L, A, Lnew, work, stream=None):
    check(lib().vb_env_left_update(mpo.h, p, mL, mR, _ptr(L), _ptr(A), _ptr(Lnew), _ptr(work),
                                   _stream_ptr(stream)))


def vb_env_right_update(mpo: Mpo, p, mL, mR, R, B, Rnew, work, stream=None):
    check(lib().vb_env_right_update(mpo.h, p, mL, mR, _ptr(R), _ptr(B), _ptr(Rnew), _ptr(work),
                                    _stream_ptr(stream)))


def vb_eig_work_bytes(n, k_want) -> int:
    return int(lib().vb_eig_work_bytes(n, k_want))


def vb_herm_eig_top(n, rho, k_want, k_vec, evals, evecs, work, stream=None):
    check(lib().vb_herm_eig_top(n, _ptr(rho), k_want, k_vec, _ptr(evals), _ptr(evecs), _ptr(work),
                                _stream_ptr(stream)))


def vb_spectrum(c_t, n_t, dt_fs, tau_fs, energies, n_e, out, stream=None):
    """Damped Fourier transform of C(t) (device buffers: c_t complex128 [n_t],
    energies float64 [n_e], out float64 [n_e])."""
    check(lib().vb_spectrum(_ptr(c_t), int(n_t), float(dt_fs), float(tau_fs), _ptr(energies), int(n_e),
                            _ptr(out), _stream_ptr(stream)))


def vb_autotune(enable: int = -1, reset: bool = False):
    """Autotuner of the tensor-core tile grouping (vb_autotune): switch it
    (1 / 0, -1 unchanged), optionally clear it; returns its table lines."""
    n = C.c_int()
    buf = C.create_string_buffer(1 << 16)
    check(lib().vb_autotune(int(enable), int(bool(reset)), C.byref(n), buf, len(buf)))
    return [x for x in buf.value.decode().splitlines() if x]


def vb_kernel_launches() -> int:
    return int(lib().vb_kernel_launches())


def vb_profile_enable(on=True, every: int = 1):
    """Switch the per-phase event profiler on (events for one call in
    `every` of each phase, times scaled) or off."""
    check(lib().vb_profile_enable(int(every) if on else 0))


def vb_profile_read(reset: bool = True) -> dict:
    p = vb_profile()
    check(lib().vb_profile_read(C.byref(p), int(reset)))
    out = {name: {"ms": p.ms[k], "calls": int(p.calls[k]), "flops": p.flops[k], "bytes": p.bytes[k]}
           for k, name in enumerate(PHASES)}
    out["heff2"]["flops"] = p.heff_flops[0]
    out["heff1"]["flops"] = p.heff_flops[1]
    out["krylov"]["flops"] = p.krylov_flops
    return out


def vb_herm_eig_top_noalloc(n, rho, k_want, k_vec, evals, evecs, stream=None):
    """vb_herm_eig_top with the library's fixed device workspace (no
    allocation; n <= 256, k_want <= 128; concurrent calls race)."""
    check(lib().vb_herm_eig_top_noalloc(n, _ptr(rho), k_want, k_vec, _ptr(evals), _ptr(evecs),
                                        _stream_ptr(stream)))


# ----------------------------------------------------------------- site order
def _order_opts(m_max, w_flops, w_size, w_coupling, iters=0, seed=0, n_strong=0):
    return vb_order_opts(int(m_max), float(w_flops), float(w_size), float(w_coupling), int(iters), int(seed),
                         int(n_strong))


def _cost_dict(c: "vb_order_cost") -> dict:
    return {"heff_flops": c.heff_flops, "tensor_elems": c.tensor_elems, "max_tensor": c.max_tensor,
            "coupling_dist": c.coupling_dist, "objective": c.objective, "max_w": c.max_w}


def site_order_cost(model: dict, order=None, m_max: int = 64, w_flops: float = 1.0, w_size: float = 1.0,
                    w_coupling: float = 1.0):
    """Cost model of a chain order (vb_site_order_cost): returns the cost
    dict, the MPO bond dimensions and the (operator, identity) block counts of
    every site."""
    keep = []
    m = _model_struct(model, keep)
    n = m.n_modes + 1
    o = _order_opts(m_max, w_flops, w_size, w_coupling)
    c = vb_order_cost()
    bonds = np.zeros(max(1, n - 1), dtype=np.int32)
    blocks = np.zeros(2 * n, dtype=np.int32)
    oa = None if order is None else np.ascontiguousarray(order, dtype=np.int32)
    check(lib().vb_site_order_cost(C.byref(m), None if oa is None else oa.ctypes.data, C.byref(o), C.byref(c),
                                   bonds.ctypes.data, blocks.ctypes.data))
    return _cost_dict(c), [int(x) for x in bonds[: n - 1]], blocks.reshape(n, 2).tolist()


def site_order_search(model: dict, m_max: int = 64, w_flops: float = 1.0, w_size: float = 1.0,
                      w_coupling: float = 1.0, iters: int = 0, seed: int = 0, n_strong: int = 0):
    """Order minimising the cost model (vb_site_order_search): returns
    (order, cost dict), order[p] = -1 for the electronic site, k for mode k."""
    keep = []
    m = _model_struct(model, keep)
    n = m.n_modes + 1
    o = _order_opts(m_max, w_flops, w_size, w_coupling, iters, seed, n_strong)
    out = np.zeros(n, dtype=np.int32)
    c = vb_order_cost()
    check(lib().vb_site_order_search(C.byref(m), C.byref(o), out.ctypes.data, C.byref(c)))
    return [int(x) for x in out], _cost_dict(c)


def site_order_rule(model: dict, n_strong: int = 4):
    """The rule-of-thumb order of vb_site_order_rule."""
    keep = []
    m = _model_struct(model, keep)
    out = np.zeros(m.n_modes + 1, dtype=np.int32)
    check(lib().vb_site_order_rule(C.byref(m), int(n_strong), out.ctypes.data))
    return [int(x) for x in out]
