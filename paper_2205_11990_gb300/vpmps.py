"""Python binding of libvpmps (ctypes; argument marshalling only).

Every operation runs in the CUDA library; this module converts numpy arrays
and torch tensors to pointers and sizes.  PyTorch supplies the CUDA stream
and, by default, device memory (its caching allocator, through the
allocator hooks of ``vp_ctx_create``).  There is no CPU fallback: without
the built library or a CUDA device the calls raise.
"""
from __future__ import annotations

import atexit
import ctypes as C
import os
import weakref

import numpy as np

from .inputs import Layout

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libvpmps.so")

VP_SEQ, VP_INTERLEAVED = 0, 1
MPO_DX_CENTERED, MPO_DX_FORWARD, MPO_DX_BACKWARD, MPO_DV_ZERO_GRAD, MPO_DXX, MPO_ADVECTION = range(6)
# contraction precision modes (vp_config.precision, vp_gemm)
PREC_FP64, PREC_FP32, PREC_TF32, PREC_BF16, PREC_TF32X3 = 0, 1, 2, 3, 4
PRECISIONS = {"fp64": PREC_FP64, "fp32": PREC_FP32, "tf32": PREC_TF32, "bf16": PREC_BF16, "tf32x3": PREC_TF32X3}

KCLASSES = ["qr_factor", "qr_formq", "gemm", "jacobi", "select", "apply", "other"]
ERRORS = {1: "VP_EINVAL", 2: "VP_ENOMEM", 3: "VP_ECAPACITY", 4: "VP_ECUDA", 5: "VP_ETIMEOUT",
          6: "VP_ENUMERIC", 7: "VP_ECFL", 8: "VP_EBUSY", 9: "VP_EIO"}

EXPORTS = [
    "vp_ctx_create", "vp_ctx_destroy", "vp_last_error", "vp_ctx_set_wait_limit", "vp_kernel_launches",
    "vp_peak_probe", "vp_profile_enable",
    "vp_profile_read", "vp_profile_trace",
    "mps_create", "mps_create_cores", "mps_destroy", "mps_num_sites", "mps_bonds", "mps_get_cores",
    "mps_to_dense", "mps_to_grid", "mps_save", "mps_load", "mps_file_info",
    "mpo_create_vp", "mpo_create_vlasov", "mpo_create_cores", "mpo_destroy", "mpo_num_sites", "mpo_bonds",
    "mpo_to_dense",
    "mps_apply_mpo", "mps_axpby", "mps_compress", "mps_compress_modified", "mps_compression_error", "vp_density", "vp_poisson", "vp_poisson_noalloc", "vp_gemm",
    "vp_sim_create", "vp_sim_destroy", "vp_step", "vp_sim_state", "vp_sim_entropy", "vp_sim_flops", "vp_run",
    "vp_footprint_bytes", "vp_batch_create", "vp_batch_submit", "vp_batch_start", "vp_batch_wait", "vp_batch_poll",
    "vp_batch_records", "vp_batch_destroy", "vp_batch_set_lockstep", "vp_batch_kernel_launches",
    "vp_multi_create", "vp_multi_destroy", "vp_multi_step", "vp_multi_state",
    "vp_group_create", "vp_group_add", "vp_group_remove", "vp_group_size", "vp_group_step", "vp_group_stats", "vp_group_mps_create", "vp_group_destroy",
]


class VpError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class CTraceRec(C.Structure):
    _fields_ = [("kclass", C.c_int), ("m", C.c_int), ("n", C.c_int), ("k", C.c_int), ("ms", C.c_double)]


class CLayout(C.Structure):
    _fields_ = [("nx", C.c_int), ("nv", C.c_int), ("mapping", C.c_int), ("xmin", C.c_double),
                ("xmax", C.c_double), ("vmin", C.c_double), ("vmax", C.c_double)]


class CConfig(C.Structure):
    _fields_ = [("dt", C.c_double), ("chi", C.c_int), ("tol", C.c_double), ("e_tol", C.c_double),
                ("streams", C.c_int), ("level", C.c_int), ("e_chi", C.c_int), ("precision", C.c_int),
                ("compression", C.c_int)]


class CSpecies(C.Structure):
    _fields_ = [("q", C.c_double), ("m", C.c_double), ("nu", C.c_double), ("u", C.c_double), ("vth", C.c_double)]


class CResult(C.Structure):
    _fields_ = [("id", C.c_uint64), ("status", C.c_int), ("nsteps", C.c_int), ("queue_ms", C.c_double),
                ("run_ms", C.c_double), ("step_ms_p50", C.c_double), ("step_ms_p99", C.c_double),
                ("field_energy", C.c_double), ("max_bond", C.c_int)]


class CRecord(C.Structure):
    _fields_ = [("t", C.c_double), ("field_energy", C.c_double), ("mass", C.c_double), ("max_bond", C.c_int),
                ("trunc_err", C.c_double)]


ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_size_t, C.c_void_p)

_lib = None
_live_contexts = weakref.WeakSet()


@atexit.register
def _close_all():
    # close while torch (whose allocator frees the memory) is still alive
    for ctx in list(_live_contexts):
        try:
            ctx.close()
        except Exception:
            pass


def load():
    """Load the shared library (raises if it was not built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libvpmps.so not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = C.CDLL(LIB_PATH)
    P, I, D, S = C.c_void_p, C.c_int, C.c_double, C.c_size_t
    DP, IP = C.POINTER(C.c_double), C.POINTER(C.c_int)
    sig = {
        "vp_ctx_create": (I, [P, ALLOC_FN, FREE_FN, P, C.POINTER(P)]),
        "vp_ctx_destroy": (I, [P]),
        "vp_last_error": (C.c_char_p, [P]),
        "vp_ctx_set_wait_limit": (I, [P, C.c_longlong]),
        "vp_peak_probe": (I, [P, I, DP]),
        "vp_kernel_launches": (C.c_int64, [P]),
        "vp_profile_enable": (I, [P, I]),
        "vp_profile_read": (I, [P, I, DP, C.POINTER(C.c_int64), DP]),
        "vp_profile_trace": (I, [P, C.POINTER(CTraceRec), I, IP]),
        "mps_create": (I, [P, C.POINTER(CLayout), P, I, I, D, C.POINTER(P)]),
        "mps_create_cores": (I, [P, I, IP, DP, C.POINTER(P)]),
        "mps_destroy": (I, [P]),
        "mps_num_sites": (I, [P]),
        "mps_bonds": (I, [P, IP]),
        "mps_get_cores": (I, [P, P, DP, S]),
        "mps_to_dense": (I, [P, P, DP]),
        "mps_to_grid": (I, [P, P, C.POINTER(CLayout), DP]),
        "mps_save": (I, [P, P, C.c_char_p]),
        "mps_load": (I, [P, C.c_char_p, C.POINTER(P)]),
        "mps_file_info": (I, [C.c_char_p, IP, IP, C.POINTER(S)]),
        "mpo_create_vp": (I, [P, C.POINTER(CLayout), I, C.POINTER(P)]),
        "mpo_create_vlasov": (I, [P, C.POINTER(CLayout), DP, D, C.POINTER(P)]),
        "mpo_create_cores": (I, [P, I, IP, DP, C.POINTER(P)]),
        "mpo_destroy": (I, [P]),
        "mpo_num_sites": (I, [P]),
        "mpo_bonds": (I, [P, IP]),
        "mpo_to_dense": (I, [P, P, DP]),
        "mps_apply_mpo": (I, [P, P, P, P]),
        "mps_axpby": (I, [P, D, P, D, P, P]),
        "mps_compress": (I, [P, P, I, D, DP]),
        "mps_compress_modified": (I, [P, P, I, I, D, DP]),
        "mps_compression_error": (I, [P, P, I, IP, D, DP]),
        "vp_density": (I, [P, C.POINTER(CLayout), P, P]),
        "vp_poisson": (I, [P, P, I, D, P, DP]),
        "vp_poisson_noalloc": (I, [P, P, I, D, P, DP, DP]),
        "vp_gemm": (I, [P, I, I, I, I, D, P, I, P, I, P, I]),
        "vp_sim_create": (I, [P, C.POINTER(CLayout), C.POINTER(CConfig), P, C.POINTER(P)]),
        "vp_sim_destroy": (I, [P]),
        "vp_step": (I, [P, I, C.POINTER(CRecord)]),
        "vp_sim_state": (P, [P]),
        "vp_sim_flops": (D, [P]),
        "vp_sim_entropy": (I, [P, DP]),
        "vp_run": (I, [P, C.POINTER(CLayout), C.POINTER(CConfig), DP, I, DP, C.POINTER(CRecord)]),
        "vp_footprint_bytes": (S, [C.POINTER(CLayout), C.POINTER(CConfig)]),
        "vp_batch_create": (I, [P, I, S, C.POINTER(P)]),
        "vp_batch_submit": (I, [P, C.POINTER(CLayout), C.POINTER(CConfig), DP, I, I, C.POINTER(C.c_uint64)]),
        "vp_batch_start": (I, [P]),
        "vp_batch_wait": (I, [P]),
        "vp_batch_poll": (I, [P, C.POINTER(CResult), I, C.POINTER(I)]),
        "vp_batch_records": (I, [P, C.c_uint64, C.POINTER(CRecord), DP, DP]),
        "vp_batch_destroy": (I, [P]),
        "vp_batch_set_lockstep": (I, [P, I]),
        "vp_batch_kernel_launches": (C.c_int64, [P]),
        "vp_multi_create": (I, [P, I, C.POINTER(CLayout), C.POINTER(CSpecies), C.POINTER(CConfig), C.POINTER(P),
                                C.POINTER(P)]),
        "vp_multi_destroy": (I, [P]),
        "vp_multi_step": (I, [P, I, C.POINTER(CRecord)]),
        "vp_multi_state": (P, [P, I]),
        "vp_group_create": (I, [P, I, C.POINTER(P)]),
        "vp_group_add": (I, [P, P]),
        "vp_group_remove": (I, [P, P]),
        "vp_group_size": (I, [P]),
        "vp_group_step": (I, [P, C.POINTER(CRecord), IP]),
        "vp_group_destroy": (I, [P]),
        "vp_group_stats": (I, [P, DP, DP, C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
        "vp_group_mps_create": (I, [P, I, C.POINTER(CLayout), C.POINTER(DP), IP, DP, C.POINTER(P), IP]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype, fn.argtypes = res, args
    _lib = lib
    return lib


def mps_file_info(path: str):
    """Validate a checkpoint file (host only, no device): (n, bond ranks,
    payload elements); raises VpError(VP_EIO) on a malformed file."""
    lib = load()
    n = C.c_int(0)
    ranks = np.zeros(65, dtype=np.int32)
    elems = C.c_size_t(0)
    st = lib.mps_file_info(os.fsencode(path), C.byref(n), _ip(ranks), C.byref(elems))
    if st != 0:
        raise VpError(st, f"mps_file_info: {path}")
    return n.value, [int(r) for r in ranks[: n.value + 1]], elems.value


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _ip(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_int))


def clayout(lay: Layout) -> CLayout:
    return CLayout(lay.nx, lay.nv, lay.mapping, lay.xmin, lay.xmax, lay.vmin, lay.vmax)


class Context:
    """A library context on torch's current CUDA stream and allocator."""

    def __init__(self, use_torch_allocator: bool = True):
        import torch
        if not torch.cuda.is_available():
            raise VpError(4, "no CUDA device")
        self.lib = load()
        self.torch = torch
        self.device = torch.cuda.current_device()
        self.stream = torch.cuda.current_stream()
        # allocation budget for failure-injection tests: None = unlimited,
        # else the number of further device allocations that may succeed
        self._budget = budget = [None]
        if use_torch_allocator:
            dev, stream = self.device, self.stream

            def _alloc(nbytes, _user):
                if budget[0] is not None:
                    if budget[0] <= 0:
                        return None
                    budget[0] -= 1
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, stream)
                except RuntimeError:
                    return None

            def _free(ptr, _nbytes, _user):
                torch.cuda.caching_allocator_delete(ptr)

            self._alloc, self._free = ALLOC_FN(_alloc), FREE_FN(_free)
        else:
            self._alloc, self._free = ALLOC_FN(), FREE_FN()
        self._children = weakref.WeakSet()
        h = C.c_void_p()
        self._check(self.lib.vp_ctx_create(C.c_void_p(self.stream.cuda_stream), self._alloc, self._free, None,
                                           C.byref(h)), ctx=None)
        self.h = h
        _live_contexts.add(self)

    def _check(self, code, ctx="self"):
        if code != 0:
            h = self.h if ctx == "self" else None
            msg = self.lib.vp_last_error(h).decode() if h is not None else "context creation failed"
            raise VpError(code, msg)

    def set_alloc_budget(self, n):
        """Let only the next n device allocations succeed (None: no limit).
        Failure injection on the host: the allocator hook returns NULL."""
        self._budget[0] = n

    PROBES = {"fp64_fma": 0, "fp32_fma": 1, "dw_dot": 2, "dw_axpy": 3, "dmma": 4}

    def peak_probe(self, kind: str) -> float:
        """Measured TFLOP/s (FP64-equivalent flops) of one unit kind."""
        out = C.c_double()
        self._check(self.lib.vp_peak_probe(self.h, self.PROBES[kind], C.byref(out)))
        return out.value

    def set_wait_limit(self, clocks: int):
        """SM clocks a device-side wait spins before giving up (0: default)."""
        self._check(self.lib.vp_ctx_set_wait_limit(self.h, int(clocks)))

    @property
    def kernel_launches(self) -> int:
        return int(self.lib.vp_kernel_launches(self.h))

    def profile(self, on: bool = True):
        self._check(self.lib.vp_profile_enable(self.h, int(on)))

    def profile_read(self):
        """{class: (ms, launches, work)} for the kernel classes timed since profile()."""
        out = {}
        for k, name in enumerate(KCLASSES):
            ms, n, w = C.c_double(), C.c_int64(), C.c_double()
            self._check(self.lib.vp_profile_read(self.h, k, C.byref(ms), C.byref(n), C.byref(w)))
            out[name] = (ms.value, int(n.value), w.value)
        return out

    def profile_trace(self):
        """Per-launch records of the profiling window: [{class, m, n, k, ms}]."""
        n = C.c_int()
        self._check(self.lib.vp_profile_trace(self.h, None, 0, C.byref(n)))
        buf = (CTraceRec * max(1, n.value))()
        self._check(self.lib.vp_profile_trace(self.h, buf, n.value, C.byref(n)))
        return [{"class": KCLASSES[r.kclass], "m": r.m, "n": r.n, "k": r.k, "ms": r.ms} for r in buf[:n.value]]

    def close(self):
        """Destroy every live MPS/MPO/Sim of this context, then the context."""
        if getattr(self, "h", None):
            for child in list(self._children):
                child.close()
            self.lib.vp_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # ------------------------------------------------------------- MPS
    def mps_from_grid(self, lay: Layout, f, chi: int, tol: float) -> "MPS":
        """a1: dense f[ix, iv] (numpy host array or CUDA torch tensor) -> MPS."""
        h = C.c_void_p()
        if isinstance(f, np.ndarray):
            f = np.ascontiguousarray(f, dtype=np.float64)
            assert f.size == lay.Nx * lay.Nv
            self._check(self.lib.mps_create(self.h, C.byref(clayout(lay)), f.ctypes.data_as(C.c_void_p), 0, chi, tol,
                                            C.byref(h)))
        else:
            assert f.is_cuda and f.dtype == self.torch.float64 and f.is_contiguous()
            self._check(self.lib.mps_create(self.h, C.byref(clayout(lay)), C.c_void_p(f.data_ptr()), 1, chi, tol,
                                            C.byref(h)))
        return MPS(self, h)

    def mps_from_cores(self, cores) -> "MPS":
        ranks = np.array([1] + [c.shape[2] for c in cores], dtype=np.int32)
        flat = np.ascontiguousarray(np.concatenate([np.asarray(c, dtype=np.float64).reshape(-1) for c in cores]))
        h = C.c_void_p()
        self._check(self.lib.mps_create_cores(self.h, len(cores), _ip(ranks), _dp(flat), C.byref(h)))
        return MPS(self, h)

    def mps_load(self, path: str) -> "MPS":
        h = C.c_void_p()
        self._check(self.lib.mps_load(self.h, os.fsencode(path), C.byref(h)))
        return MPS(self, h)

    def mpo_vp(self, lay: Layout, kind: int) -> "MPO":
        h = C.c_void_p()
        self._check(self.lib.mpo_create_vp(self.h, C.byref(clayout(lay)), kind, C.byref(h)))
        return MPO(self, h)

    def mpo_vlasov(self, lay: Layout, E: np.ndarray, e_tol: float) -> "MPO":
        E = np.ascontiguousarray(E, dtype=np.float64)
        h = C.c_void_p()
        self._check(self.lib.mpo_create_vlasov(self.h, C.byref(clayout(lay)), _dp(E), e_tol, C.byref(h)))
        return MPO(self, h)

    def mpo_from_cores(self, cores) -> "MPO":
        bonds = np.array([1] + [c.shape[3] for c in cores], dtype=np.int32)
        flat = np.ascontiguousarray(np.concatenate([np.asarray(c, dtype=np.float64).reshape(-1) for c in cores]))
        h = C.c_void_p()
        self._check(self.lib.mpo_create_cores(self.h, len(cores), _ip(bonds), _dp(flat), C.byref(h)))
        return MPO(self, h)

    def empty_mps(self) -> "MPS":
        return self.mps_from_cores([np.zeros((1, 2, 1))])

    # ------------------------------------------------------- operations
    def apply_mpo(self, mpo: "MPO", x: "MPS", out: "MPS" = None) -> "MPS":
        out = out or self.empty_mps()
        self._check(self.lib.mps_apply_mpo(self.h, mpo.h, x.h, out.h))
        return out

    def axpby(self, a: float, x: "MPS", b: float, y: "MPS", out: "MPS" = None) -> "MPS":
        out = out or self.empty_mps()
        self._check(self.lib.mps_axpby(self.h, a, x.h, b, y.h, out.h))
        return out

    def compress(self, x: "MPS", chi: int, tol: float) -> np.ndarray:
        errs = np.zeros(max(1, x.n - 1))
        self._check(self.lib.mps_compress(self.h, x.h, chi, tol, _dp(errs)))
        return errs[: x.n - 1]

    def compression_error(self, x: "MPS", chis, tol: float = 0.0) -> np.ndarray:
        """rms over the grid of f - f_D for each bond cap D in chis."""
        ch = np.ascontiguousarray(chis, dtype=np.int32)
        out = np.zeros(len(ch))
        self._check(self.lib.mps_compression_error(self.h, x.h, len(ch), _ip(ch), tol, _dp(out)))
        return out

    def compress_modified(self, x: "MPS", split: int, chi: int, tol: float) -> np.ndarray:
        errs = np.zeros(max(1, x.n - 1))
        self._check(self.lib.mps_compress_modified(self.h, x.h, split, chi, tol, _dp(errs)))
        return errs[: x.n - 1]

    def density(self, lay: Layout, f: "MPS"):
        rho = self.torch.empty(lay.Nx, dtype=self.torch.float64, device="cuda")
        self._check(self.lib.vp_density(self.h, C.byref(clayout(lay)), f.h, C.c_void_p(rho.data_ptr())))
        return rho

    def poisson(self, rho, nx: int, dx: float):
        E = self.torch.empty(1 << nx, dtype=self.torch.float64, device="cuda")
        we = C.c_double()
        self._check(self.lib.vp_poisson(self.h, C.c_void_p(rho.data_ptr()), nx, dx, C.c_void_p(E.data_ptr()),
                                        C.byref(we)))
        return E, we.value

    def poisson_noalloc(self, rho, nx: int, dx: float, E=None):
        """vp_poisson_noalloc on this context's stream (no context memory used)."""
        E = E if E is not None else self.torch.empty(1 << nx, dtype=self.torch.float64, device="cuda")
        we, mass = C.c_double(), C.c_double()
        code = self.lib.vp_poisson_noalloc(C.c_void_p(self.stream.cuda_stream), C.c_void_p(rho.data_ptr()), nx, dx,
                                           C.c_void_p(E.data_ptr()), C.byref(we), C.byref(mass))
        if code != 0:
            raise VpError(code, "vp_poisson_noalloc failed")
        return E, we.value, mass.value

    def gemm(self, A, B, alpha: float = 1.0, precision: int = 0):
        """vp_gemm: alpha * A @ B for 2-D float64 CUDA tensors (row-major)."""
        t = self.torch
        A = A.contiguous()
        B = B.contiguous()
        M, K = A.shape
        K2, N = B.shape
        if K2 != K:
            raise ValueError("gemm: inner dimensions differ")
        Cout = t.empty((M, N), dtype=t.float64, device=A.device)
        self._check(self.lib.vp_gemm(self.h, precision, M, N, K, alpha, C.c_void_p(A.data_ptr()), max(K, 1),
                                     C.c_void_p(B.data_ptr()), max(N, 1), C.c_void_p(Cout.data_ptr()), max(N, 1)))
        return Cout

    def sim(self, lay: Layout, f0: "MPS", dt: float, chi: int, tol: float = 1e-10, e_tol: float = 1e-10,
            streams: int = 2, level: int = 1, e_chi: int = 0, precision: int = 0, compression: int = 0) -> "Sim":
        h = C.c_void_p()
        cfg = CConfig(dt, chi, tol, e_tol, streams, level, e_chi, precision, compression)
        self._check(self.lib.vp_sim_create(self.h, C.byref(clayout(lay)), C.byref(cfg), f0.h, C.byref(h)))
        return Sim(self, h, lay)

    def group(self, max_members: int) -> "Group":
        return Group(self, max_members)

    def multi(self, lays, species, f0s, dt: float, chi: int, tol: float = 1e-10, e_tol: float = 1e-10,
              streams: int = 2, e_chi: int = 0, precision: int = 0, compression: int = 0) -> "Multi":
        """Several species sharing one field (vp_multi_*).  species: per
        species (q, m) or (q, m, nu, u, vth); f0s: per species an MPS."""
        ns = len(lays)
        if not (len(species) == len(f0s) == ns):
            raise ValueError("multi: one layout, species and initial state per species")
        cl = (CLayout * ns)(*[clayout(l) for l in lays])
        sp = []
        for t in species:
            t = tuple(t) + (0.0, 0.0, 1.0)[len(t) - 2:] if len(t) < 5 else tuple(t)
            sp.append(CSpecies(*[float(x) for x in t]))
        cs = (CSpecies * ns)(*sp)
        fp = (C.c_void_p * ns)(*[f.h for f in f0s])
        cfg = CConfig(dt, chi, tol, e_tol, streams, 1, e_chi, precision, compression)
        h = C.c_void_p()
        self._check(self.lib.vp_multi_create(self.h, ns, cl, cs, C.byref(cfg), fp, C.byref(h)))
        return Multi(self, h, list(lays))

    def run(self, lay: Layout, f0: np.ndarray, dt: float, nsteps: int, chi: int, tol: float = 1e-10,
            e_tol: float = 1e-10, want_f: bool = True, streams: int = 2):
        f0 = np.ascontiguousarray(f0, dtype=np.float64)
        fT = np.zeros((lay.Nx, lay.Nv)) if want_f else None
        recs = (CRecord * max(1, nsteps))()
        cfg = CConfig(dt, chi, tol, e_tol, streams, 1, 0, 0)
        self._check(self.lib.vp_run(self.h, C.byref(clayout(lay)), C.byref(cfg), _dp(f0), nsteps,
                                    _dp(fT) if want_f else None, recs))
        return fT, _records(recs, nsteps)


class Batch:
    """Concurrent independent runs (vp_batch_*): submit, start, wait/poll.
    lockstep=G > 0: G workers, each stepping its resident runs (one site
    count per worker) as one lockstep group (continuous batching); else one
    worker thread per run."""

    def __init__(self, ctx: Context, max_concurrent: int, mem_budget_bytes: int, lockstep: int = 0):
        self.ctx = ctx
        h = C.c_void_p()
        ctx._check(ctx.lib.vp_batch_create(ctx.h, max_concurrent, mem_budget_bytes, C.byref(h)))
        self.h = h
        if lockstep:
            ctx._check(ctx.lib.vp_batch_set_lockstep(h, int(lockstep)))
        self.nsteps = {}
        ctx._children.add(self)

    def submit(self, lay: Layout, f0: np.ndarray, dt: float, nsteps: int, chi: int, tol: float = 1e-10,
               e_tol: float = 1e-10, keep_f: bool = False) -> int:
        f0 = np.ascontiguousarray(f0, dtype=np.float64)
        rid = C.c_uint64()
        cfg = CConfig(dt, chi, tol, e_tol, 1, 1, 0, 0)
        self.ctx._check(self.ctx.lib.vp_batch_submit(self.h, C.byref(clayout(lay)), C.byref(cfg), _dp(f0), nsteps,
                                                     int(keep_f), C.byref(rid)))
        self.nsteps[rid.value] = (nsteps, lay)
        return rid.value

    def start(self):
        self.ctx._check(self.ctx.lib.vp_batch_start(self.h))

    def wait(self):
        self.ctx._check(self.ctx.lib.vp_batch_wait(self.h))

    def poll(self, max_n: int = 1024):
        out = (CResult * max_n)()
        n = C.c_int()
        self.ctx._check(self.ctx.lib.vp_batch_poll(self.h, out, max_n, C.byref(n)))
        return [{k: getattr(r, k) for k, _ in CResult._fields_} for r in list(out)[: n.value]]

    def records(self, rid: int, want_f: bool = False):
        nsteps, lay = self.nsteps[rid]
        recs = (CRecord * max(1, nsteps))()
        ms = np.zeros(max(1, nsteps))
        fT = np.zeros((lay.Nx, lay.Nv)) if want_f else None
        self.ctx._check(self.ctx.lib.vp_batch_records(self.h, rid, recs, _dp(ms), _dp(fT) if want_f else None))
        return _records(recs, nsteps), ms[:nsteps], fT

    @property
    def kernel_launches(self) -> int:
        """Kernels launched by the batch's worker contexts (read while they are idle)."""
        return int(self.ctx.lib.vp_batch_kernel_launches(self.h)) if self.h else 0

    def close(self):
        if self.h and self.ctx.h:
            self.ctx.lib.vp_batch_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def footprint_bytes(lay: Layout, chi: int, dt: float = 0.01) -> int:
    return int(load().vp_footprint_bytes(C.byref(clayout(lay)), C.byref(CConfig(dt, chi, 1e-10, 1e-10, 1, 1, 0, 0))))


def _records(recs, n):
    return [dict(t=r.t, field_energy=r.field_energy, mass=r.mass, max_bond=r.max_bond, trunc_err=r.trunc_err)
            for r in list(recs)[:n]]


class MPS:
    def __init__(self, ctx: Context, h, owned: bool = True):
        self.ctx, self.h, self.owned = ctx, h, owned
        ctx._children.add(self)

    @property
    def n(self) -> int:
        return int(self.ctx.lib.mps_num_sites(self.h))

    def bonds(self):
        out = np.zeros(self.n + 1, dtype=np.int32)
        self.ctx._check(self.ctx.lib.mps_bonds(self.h, _ip(out)))
        return [int(x) for x in out]

    def cores(self):
        r = self.bonds()
        sizes = [r[k] * 2 * r[k + 1] for k in range(self.n)]
        flat = np.zeros(sum(sizes))
        self.ctx._check(self.ctx.lib.mps_get_cores(self.ctx.h, self.h, _dp(flat), flat.size))
        out, off = [], 0
        for k, s in enumerate(sizes):
            out.append(flat[off:off + s].reshape(r[k], 2, r[k + 1]))
            off += s
        return out

    def save(self, path: str) -> None:
        self.ctx._check(self.ctx.lib.mps_save(self.ctx.h, self.h, os.fsencode(path)))

    def to_dense(self) -> np.ndarray:
        out = np.zeros(1 << self.n)
        self.ctx._check(self.ctx.lib.mps_to_dense(self.ctx.h, self.h, _dp(out)))
        return out

    def to_grid(self, lay: Layout) -> np.ndarray:
        out = np.zeros((lay.Nx, lay.Nv))
        self.ctx._check(self.ctx.lib.mps_to_grid(self.ctx.h, self.h, C.byref(clayout(lay)), _dp(out)))
        return out

    def close(self):
        if self.owned and self.h and self.ctx.h:
            self.ctx.lib.mps_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class MPO:
    def __init__(self, ctx: Context, h):
        self.ctx, self.h = ctx, h
        ctx._children.add(self)

    @property
    def n(self) -> int:
        return int(self.ctx.lib.mpo_num_sites(self.h))

    def bonds(self):
        out = np.zeros(self.n + 1, dtype=np.int32)
        self.ctx._check(self.ctx.lib.mpo_bonds(self.h, _ip(out)))
        return [int(x) for x in out]

    def to_dense(self) -> np.ndarray:
        n = self.n
        out = np.zeros((1 << n, 1 << n))
        self.ctx._check(self.ctx.lib.mpo_to_dense(self.ctx.h, self.h, _dp(out)))
        return out

    def close(self):
        if self.h and self.ctx.h:
            self.ctx.lib.mpo_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Sim:
    def __init__(self, ctx: Context, h, lay: Layout):
        self.ctx, self.h, self.lay = ctx, h, lay
        ctx._children.add(self)

    def step(self, nsteps: int = 1):
        recs = (CRecord * max(1, nsteps))()
        self.ctx._check(self.ctx.lib.vp_step(self.h, nsteps, recs))
        return _records(recs, nsteps)

    def state(self) -> MPS:
        return MPS(self.ctx, C.c_void_p(self.ctx.lib.vp_sim_state(self.h)), owned=False)

    @property
    def flops(self) -> float:
        return float(self.ctx.lib.vp_sim_flops(self.h))

    def entropy(self) -> np.ndarray:
        out = np.zeros(max(1, self.lay.n - 1))
        self.ctx._check(self.ctx.lib.vp_sim_entropy(self.h, _dp(out)))
        return out[: self.lay.n - 1]

    def close(self):
        if self.h and self.ctx.h:
            self.ctx.lib.vp_sim_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Group:
    """Simulations stepped in lockstep, every launch serving all members
    (vp_group_*).  Members: sims of this context created with streams=1."""

    def __init__(self, ctx: Context, max_members: int):
        self.ctx = ctx
        h = C.c_void_p()
        ctx._check(ctx.lib.vp_group_create(ctx.h, max_members, C.byref(h)))
        self.h = h
        self.members = []
        ctx._children.add(self)

    def add(self, sim: "Sim"):
        self.ctx._check(self.ctx.lib.vp_group_add(self.h, sim.h))
        self.members.append(sim)

    def remove(self, sim: "Sim"):
        self.ctx._check(self.ctx.lib.vp_group_remove(self.h, sim.h))
        self.members.remove(sim)

    def __len__(self):
        return int(self.ctx.lib.vp_group_size(self.h))

    def step(self):
        """One step of every running member: (records, status) per member."""
        n = len(self.members)
        recs = (CRecord * max(1, n))()
        st = np.zeros(max(1, n), dtype=np.int32)
        self.ctx._check(self.ctx.lib.vp_group_step(self.h, recs, _ip(st)))
        return _records(recs, n), [int(x) for x in st[:n]]

    def create_mps(self, items):
        """Batched a1: items = [(layout, f host grid, chi, tol)] -> ([MPS or
        None], [status]) as mps_create would make each."""
        n = len(items)
        lays = (CLayout * max(1, n))(*[clayout(l) for l, _, _, _ in items])
        grids = [np.ascontiguousarray(f, dtype=np.float64) for _, f, _, _ in items]
        fptr = (C.POINTER(C.c_double) * max(1, n))(*[_dp(gr) for gr in grids])
        chis = np.array([c for _, _, c, _ in items], dtype=np.int32)
        tols = np.array([t for _, _, _, t in items], dtype=np.float64)
        outs = (C.c_void_p * max(1, n))()
        st = np.zeros(max(1, n), dtype=np.int32)
        self.ctx._check(self.ctx.lib.vp_group_mps_create(self.h, n, lays, fptr, _ip(chis), _dp(tols), outs, _ip(st)))
        return [MPS(self.ctx, C.c_void_p(h)) if h else None for h in outs[:n]], [int(x) for x in st[:n]]

    def stats(self):
        """Last step: host wall ms, ms waiting for the device, waits, launches."""
        a, b, c, d = C.c_double(), C.c_double(), C.c_int64(), C.c_int64()
        self.ctx._check(self.ctx.lib.vp_group_stats(self.h, C.byref(a), C.byref(b), C.byref(c), C.byref(d)))
        return {"step_ms": a.value, "wait_ms": b.value, "waits": c.value, "launches": d.value}

    def close(self):
        if self.h and self.ctx.h:
            self.ctx.lib.vp_group_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Multi:
    """Several species advanced in lockstep on one field (vp_multi_*)."""

    def __init__(self, ctx: Context, h, lays):
        self.ctx, self.h, self.lays = ctx, h, lays
        ctx._children.add(self)

    def step(self, nsteps: int = 1):
        """Per step: t, the shared field energy, and per species mass,
        max bond and truncation error (lists)."""
        ns = len(self.lays)
        recs = (CRecord * max(1, nsteps * ns))()
        self.ctx._check(self.ctx.lib.vp_multi_step(self.h, nsteps, recs))
        out = []
        for n in range(nsteps):
            r = [recs[n * ns + s] for s in range(ns)]
            out.append(dict(t=r[0].t, field_energy=r[0].field_energy, mass=[x.mass for x in r],
                            max_bond=[x.max_bond for x in r], trunc_err=[x.trunc_err for x in r]))
        return out

    def state(self, s: int) -> MPS:
        p = self.ctx.lib.vp_multi_state(self.h, s)
        if not p:
            raise IndexError(s)
        return MPS(self.ctx, C.c_void_p(p), owned=False)

    def close(self):
        if self.h and self.ctx.h:
            self.ctx.lib.vp_multi_destroy(self.h)
        self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
