"""Python binding of ``libqcs`` (the C ABI in ``include/qcs.h``).

Argument marshalling only: every step of the overlap path runs in the CUDA
kernels of ``libqcs.so``.  Tensors are PyTorch CUDA tensors (complex128 for
walkers, overlaps and gradients; float64 for Q; uint8 for b); the current
PyTorch stream is passed to the library.  There is no CPU fallback: if the
library cannot be loaded, or no CUDA device is present, these functions
raise.
"""
from __future__ import annotations

import ctypes
import json
import os
import threading

import torch

from . import _build

_lib = None
_lock = threading.Lock()

QCS_OK = 0
QCS_FP64 = 0
QCS_TF32X3 = 1
QCS_FLAG_ALL_NODES = 1
QCS_FLAG_DFT_NODES = 2
QCS_FLAG_FP64_ALU = 4
QCS_FLAG_FP64_TC = 8
MAX_NODES = 49
QCS_ERR_ARG, QCS_ERR_CUDA, QCS_ERR_NONFINITE, QCS_ERR_SINGULAR, QCS_ERR_TIMEOUT, QCS_ERR_UNSUPPORTED = 1, 2, 4, 8, 16, 32
QCS_ERR_BOUNDS = 64
STATUS_BITS = {1: "ARG", 2: "CUDA", 4: "NONFINITE", 8: "SINGULAR", 16: "TIMEOUT", 32: "UNSUPPORTED"}

EXPORTED = [
    "qcs_create", "qcs_destroy", "qcs_last_error", "qcs_sync_status", "qcs_workspace_bytes",
    "qcs_build_snapshots", "qcs_snapshots_free", "qcs_snapshots_parity", "qcs_snapshots_count",
    "qcs_snapshots_modes", "qcs_overlap", "qcs_overlap_grad", "qcs_force_bias", "qcs_overlap_flops_per_pair",
    "qcs_profile_enable", "qcs_profile_read", "qcs_grad_flops_per_pair", "qcs_overlap_noalloc",
    "qcs_autotune", "qcs_set_config", "qcs_overlap_batched", "qcs_node_plan_get",
    "qcs_snapshots_signed_perm_count", "qcs_overlap_flops_per_pair_signed_perm",
    "qcs_grad_flops_per_pair_signed_perm", "qcs_shadow_rdm", "qcs_shadow_rdm_flops", "qcs_vce_transform",
    "qcs_local_energy", "qcs_local_energy_flops_per_pair", "qcs_overlap_flops_breakdown",
    "qcs_selftest_bounded_wait", "qcs_fp64_fma_rate", "qcs_overlap_tc_work_per_pair", "qcs_set_allocator",
    "qcs_selftest_reciprocal",
]
MAX_SYSTEMS = 8
TUNE_CACHE = os.environ.get("QCS_TUNE_CACHE", os.path.join(os.path.expanduser("~"), ".cache", "qcs", "tune.json"))
NOALLOC_SCRATCH_BYTES = 32 << 20


_ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
_FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)


class QCSError(RuntimeError):
    def __init__(self, code, msg):
        names = [v for k, v in STATUS_BITS.items() if code & k]
        super().__init__(f"libqcs error {code} ({'|'.join(names) or 'OK'}): {msg}")
        self.code = code


class _System(ctypes.Structure):
    _fields_ = [("snapshots", ctypes.c_void_p), ("ne", ctypes.c_int), ("W", ctypes.c_int64),
                ("d_walkers", ctypes.c_void_p), ("d_overlap", ctypes.c_void_p)]


class _Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("nodes", ctypes.c_int), ("flags", ctypes.c_uint),
                ("config", ctypes.c_int)]


def decode_config(config: int) -> dict:
    """The fields of a kernel configuration (qcs_opts.config); 0 in a field = default."""
    c = int(config)
    return {"node_matrices_per_round": c & 15, "alu_snapshots_per_warp": (c >> 4) & 15,
            "alu_warps_per_pair": (c >> 8) & 3, "path": {0: "default", 1: "fp64_alu", 2: "tensor_cores"}[(c >> 10) & 3],
            "tc_subtiles_per_tile": (c >> 12) & 15}


def encode_config(node_matrices_per_round=0, alu_snapshots_per_warp=0, alu_warps_per_pair=0, path=0,
                  tc_subtiles_per_tile=0) -> int:
    """qcs_opts.config from its fields (path: 0 default, 1 FP64 ALU, 2 tensor cores)."""
    return ((node_matrices_per_round & 15) | (alu_snapshots_per_warp & 15) << 4 | (alu_warps_per_pair & 3) << 8
            | (path & 3) << 10 | (tc_subtiles_per_tile & 15) << 12)


def library_path() -> str:
    """The library this process loads: libqcs.so in the source tree, or what the
    environment variable QCS_LIBRARY names ("bounds" for the bounds-checked debug build
    libqcs_bounds.so, built in-tree on first use; otherwise a path to a libqcs build)."""
    sel = os.environ.get("QCS_LIBRARY", "")
    if sel == "bounds":
        return _build.lib_path("bounds")
    return sel or _build.LIB


def load(build_if_missing: bool = True):
    """Load libqcs.so (building it in-tree with nvcc if missing or stale)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = library_path()
        sel = os.environ.get("QCS_LIBRARY", "")
        if build_if_missing and sel in ("", "bounds") and _build.stale(sel or None):
            _build.build(variant=sel or None)
        if not os.path.exists(path):
            raise RuntimeError(f"libqcs.so not found at {path}; run __graft_entry__.build()")
        lib = ctypes.CDLL(path)
        P, i32, i64, u32, f64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint, ctypes.c_double
        lib.qcs_create.argtypes = [ctypes.POINTER(P), i32]
        lib.qcs_destroy.argtypes = [P]
        lib.qcs_last_error.argtypes = [P]
        lib.qcs_last_error.restype = ctypes.c_char_p
        lib.qcs_sync_status.argtypes = [P, P]
        lib.qcs_workspace_bytes.argtypes = [P]
        lib.qcs_workspace_bytes.restype = ctypes.c_size_t
        lib.qcs_selftest_bounded_wait.argtypes = [P, u32, P]
        lib.qcs_selftest_reciprocal.argtypes = [P, P, P, i64, P]
        lib.qcs_fp64_fma_rate.argtypes = [P, ctypes.POINTER(f64), P]
        lib.qcs_overlap_tc_work_per_pair.argtypes = [i32, i32, i32, u32, ctypes.POINTER(f64), ctypes.POINTER(f64)]
        lib.qcs_set_allocator.argtypes = [P, _ALLOC_FN, _FREE_FN, P]
        lib.qcs_build_snapshots.argtypes = [P, i32, i64, P, P, ctypes.POINTER(P), P]
        lib.qcs_snapshots_free.argtypes = [P]
        lib.qcs_snapshots_parity.argtypes = [P, P, P]
        lib.qcs_snapshots_count.argtypes = [P]
        lib.qcs_snapshots_count.restype = i64
        lib.qcs_snapshots_modes.argtypes = [P]
        lib.qcs_overlap.argtypes = [P, P, i32, i64, P, P, P, ctypes.POINTER(_Opts), P]
        lib.qcs_overlap_grad.argtypes = [P, P, i32, i64, P, P, P, ctypes.POINTER(_Opts), P]
        lib.qcs_force_bias.argtypes = [P, i32, i32, i64, i32, P, P, P, P, f64, P, P]
        lib.qcs_overlap_flops_per_pair.argtypes = [i32, i32, i32, u32]
        lib.qcs_overlap_flops_per_pair.restype = f64
        lib.qcs_grad_flops_per_pair.argtypes = [i32, i32, i32, u32]
        lib.qcs_grad_flops_per_pair.restype = f64
        lib.qcs_node_plan_get.argtypes = [i32, i32, i32, u32, ctypes.POINTER(i32), P, P]
        lib.qcs_snapshots_signed_perm_count.argtypes = [P, ctypes.POINTER(i64), P]
        lib.qcs_shadow_rdm.argtypes = [P, P, P, P, P, P, P, P]
        lib.qcs_vce_transform.argtypes = [P, i32, i32, i32, i32, i64, P, P, i64, i32, P, P]
        lib.qcs_local_energy.argtypes = [P, P, i32, i64, P, i32, P, P, P, P, P, ctypes.POINTER(_Opts), P]
        lib.qcs_local_energy_flops_per_pair.argtypes = [i32, i32, i32, i32, i32, u32]
        lib.qcs_local_energy_flops_per_pair.restype = f64
        lib.qcs_shadow_rdm_flops.argtypes = [i32, i64]
        lib.qcs_shadow_rdm_flops.restype = f64
        for fn in ("qcs_overlap_flops_per_pair_signed_perm", "qcs_grad_flops_per_pair_signed_perm"):
            getattr(lib, fn).argtypes = [i32, i32, i32, u32]
            getattr(lib, fn).restype = f64
        lib.qcs_overlap_flops_breakdown.argtypes = [i32, i32, i32, u32, ctypes.POINTER(f64)]
        lib.qcs_overlap_batched.argtypes = [P, i32, ctypes.POINTER(_System), ctypes.POINTER(_Opts), P]
        lib.qcs_autotune.argtypes = [P, i32, i32, i32, u32, ctypes.POINTER(i32)]
        lib.qcs_set_config.argtypes = [P, i32, i32, i32, u32, i32]
        lib.qcs_overlap_noalloc.argtypes = [i32, i32, i64, P, P, i64, P, P, P, P]
        lib.qcs_profile_enable.argtypes = [P, i32]
        lib.qcs_profile_read.argtypes = [P, ctypes.POINTER(f64), ctypes.POINTER(i64)]
        _lib = lib
        return lib


def _stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _need_cuda(t, name, dtype):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


class Context:
    """A libqcs context on one CUDA device (owns the workspace and status word)."""

    def __init__(self, device: int | None = None):
        if not torch.cuda.is_available():
            raise RuntimeError("libqcs needs a CUDA device; none is visible")
        self.lib = load()
        self.device = torch.cuda.current_device() if device is None else int(device)
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            rc = self.lib.qcs_create(ctypes.byref(h), self.device)
        if rc != QCS_OK:
            raise QCSError(rc, "qcs_create failed")
        self.h = h
        self.gpu_name = torch.cuda.get_device_name(self.device)
        for key, cfg in _read_cache().get(self.gpu_name, {}).items():
            n, ne, nodes, flags = (int(x) for x in key.split(","))
            self.lib.qcs_set_config(self.h, n, ne, nodes, flags, int(cfg))

    def autotune(self, n: int, ne: int, nodes: int = 0, flags: int = 0, save: bool = True,
                 use_cache: bool = False) -> int:
        """Time the pair-kernel configurations for these sizes on this GPU, keep the
        fastest in the context, and (save=True) record it in the tuning cache.  With
        use_cache=True a choice already in the cache for this GPU is taken as is
        (it was loaded into the context when the context was created)."""
        if use_cache:
            hit = _read_cache().get(self.gpu_name, {}).get(f"{n},{ne},{nodes},{flags}")
            if hit is not None:
                return int(hit)
        cfg = ctypes.c_int()
        self.check(self.lib.qcs_autotune(self.h, n, ne, nodes, flags, ctypes.byref(cfg)))
        if save:
            cache = _read_cache()
            cache.setdefault(self.gpu_name, {})[f"{n},{ne},{nodes},{flags}"] = cfg.value
            try:
                os.makedirs(os.path.dirname(TUNE_CACHE), exist_ok=True)
                tmp = TUNE_CACHE + f".tmp{os.getpid()}"
                with open(tmp, "w") as f:
                    json.dump(cache, f, indent=1, sort_keys=True)
                os.replace(tmp, TUNE_CACHE)
            except OSError:
                pass
        return cfg.value

    def set_config(self, n: int, ne: int, config: int, nodes: int = 0, flags: int = 0):
        self.check(self.lib.qcs_set_config(self.h, n, ne, nodes, flags, config))

    def check(self, rc):
        if rc != QCS_OK:
            raise QCSError(rc, self.lib.qcs_last_error(self.h).decode())

    def sync_status(self) -> int:
        return int(self.lib.qcs_sync_status(self.h, _stream()))

    def workspace_bytes(self) -> int:
        return int(self.lib.qcs_workspace_bytes(self.h))

    def selftest_bounded_wait(self, max_iter: int = 64) -> int:
        """Run the device time-out self-test; returns the status bits it raised."""
        self.check(self.lib.qcs_selftest_bounded_wait(self.h, max_iter, _stream()))
        return self.sync_status()

    def selftest_reciprocal(self, d):
        """r = 1/d through the eliminations' pivot reciprocal (qcs_selftest_reciprocal);
        d a float64 CUDA tensor of values >= 0 on this context's device."""
        import torch

        if d.dtype != torch.float64 or not d.is_cuda or d.device.index != self.device:
            raise ValueError("d must be a float64 tensor on the context's device")
        d = d.contiguous()
        r = torch.empty_like(d)
        with torch.cuda.device(self.device):
            self.check(self.lib.qcs_selftest_reciprocal(self.h, _ptr(d), _ptr(r), d.numel(), _stream()))
        return r

    def use_torch_allocator(self):
        """Back the context's device memory (workspace, snapshot sets built afterwards,
        tensor-core records, the autotuner's sample) with PyTorch's caching allocator
        (qcs_set_allocator).  alloc_calls / free_calls count the callbacks."""
        dev = self.device
        self.alloc_calls = 0
        self.free_calls = 0

        def _alloc(nbytes, stream, user):
            try:
                self.alloc_calls += 1
                return torch.cuda.caching_allocator_alloc(int(nbytes), device=dev, stream=int(stream or 0))
            except Exception:  # the library reports QCS_ERR_CUDA for a NULL result
                return None

        def _free(ptr, nbytes, stream, user):
            self.free_calls += 1
            torch.cuda.caching_allocator_delete(ptr)

        cbs = (_ALLOC_FN(_alloc), _FREE_FN(_free))
        self.check(self.lib.qcs_set_allocator(self.h, cbs[0], cbs[1], None))
        self._allocator_callbacks = cbs  # kept alive as long as the context (and its snapshot sets)

    def use_cuda_malloc(self):
        """Back later device memory with cudaMalloc again (snapshot sets already built keep
        the allocator they were built with, and the callbacks stay alive for them)."""
        self.check(self.lib.qcs_set_allocator(self.h, _ALLOC_FN(), _FREE_FN(), None))

    def fp64_fma_rate(self) -> float:
        """Sustained FP64 FMA rate of this device in TFLOP/s (about 2.5 s of chains)."""
        t = ctypes.c_double()
        self.check(self.lib.qcs_fp64_fma_rate(self.h, ctypes.byref(t), _stream()))
        return float(t.value)

    def profile(self, enable: bool = True):
        self.check(self.lib.qcs_profile_enable(self.h, 1 if enable else 0))

    def profile_read(self):
        """(summed milliseconds, launches) of the dominant kernels since the last read."""
        ms, n = ctypes.c_double(), ctypes.c_int64()
        self.check(self.lib.qcs_profile_read(self.h, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def close(self):
        if getattr(self, "h", None):
            self.lib.qcs_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _read_cache() -> dict:
    try:
        with open(TUNE_CACHE) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


class Snapshots:
    """Device-resident snapshot set built by qcs_build_snapshots."""

    def __init__(self, ctx: Context, Q: torch.Tensor, b: torch.Tensor):
        _need_cuda(Q, "Q", torch.float64)
        _need_cuda(b, "b", torch.uint8)
        P, N, N2 = Q.shape
        n = N // 2
        if N != N2 or N != 2 * n or tuple(b.shape) != (P, n):
            raise ValueError("Q must be (P, 2n, 2n) and b (P, n)")
        self.ctx, self.n, self.P = ctx, n, P
        h = ctypes.c_void_p()
        ctx.check(ctx.lib.qcs_build_snapshots(ctx.h, n, P, _ptr(Q), _ptr(b), ctypes.byref(h), _stream()))
        self.h = h

    def parity(self) -> torch.Tensor:
        out = torch.empty(self.P, dtype=torch.int8, device=f"cuda:{self.ctx.device}")
        self.ctx.check(self.ctx.lib.qcs_snapshots_parity(self.h, _ptr(out), _stream()))
        return out

    def signed_perm_count(self) -> int:
        """Snapshots of the set that are signed permutations (gather path); waits for
        the current stream."""
        c = ctypes.c_int64(0)
        self.ctx.check(self.ctx.lib.qcs_snapshots_signed_perm_count(self.h, ctypes.byref(c), _stream()))
        return int(c.value)

    def close(self):
        if getattr(self, "h", None):
            self.ctx.lib.qcs_snapshots_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _opts(nodes=0, flags=0, precision=QCS_FP64, config=0):
    return _Opts(int(precision), int(nodes), int(flags), int(config))


def overlap(ctx: Context, snaps: Snapshots, walkers: torch.Tensor, per_pair: bool = False, nodes: int = 0,
            flags: int = 0, precision: int = QCS_FP64, config: int = 0):
    """<Psi_T|phi_w> for walkers (W, n, ne) complex128; returns (overlap[W], per_pair[W, P] or None)."""
    _need_cuda(walkers, "walkers", torch.complex128)
    W, n, ne = walkers.shape
    if n != snaps.n:
        raise ValueError("walker size does not match the snapshot set")
    dev = walkers.device
    out = torch.empty(W, dtype=torch.complex128, device=dev)
    pp = torch.empty((W, snaps.P), dtype=torch.complex128, device=dev) if per_pair else None
    o = _opts(nodes, flags, precision, config)
    ctx.check(ctx.lib.qcs_overlap(ctx.h, snaps.h, ne, W, _ptr(walkers), _ptr(out), _ptr(pp), ctypes.byref(o),
                                  _stream()))
    return out, pp


def overlap_batched(ctx: Context, systems, nodes: int = 0, flags: int = 0, outs=None):
    """Overlaps of several systems [(snaps, walkers), ...] in one pair-kernel launch.
    Returns a list of overlap tensors (or fills ``outs``)."""
    if not 1 <= len(systems) <= MAX_SYSTEMS:
        raise ValueError(f"1..{MAX_SYSTEMS} systems")
    arr = (_System * len(systems))()
    res = []
    for i, (snaps, walkers) in enumerate(systems):
        _need_cuda(walkers, "walkers", torch.complex128)
        W, n, ne = walkers.shape
        if n != snaps.n:
            raise ValueError("walker size does not match its snapshot set")
        out = outs[i] if outs is not None else torch.empty(W, dtype=torch.complex128, device=walkers.device)
        arr[i] = _System(snaps.h.value, ne, W, walkers.data_ptr(), out.data_ptr())
        res.append(out)
    o = _opts(nodes, flags)
    ctx.check(ctx.lib.qcs_overlap_batched(ctx.h, len(systems), arr, ctypes.byref(o), _stream()))
    return res


def overlap_grad(ctx: Context, snaps: Snapshots, walkers: torch.Tensor, nodes: int = 0, flags: int = 0):
    """(overlap[W], grad[W, n, ne]) with grad = d overlap / d walkers (holomorphic)."""
    _need_cuda(walkers, "walkers", torch.complex128)
    W, n, ne = walkers.shape
    dev = walkers.device
    out = torch.empty(W, dtype=torch.complex128, device=dev)
    g = torch.empty((W, n, ne), dtype=torch.complex128, device=dev)
    o = _opts(nodes, flags)
    ctx.check(ctx.lib.qcs_overlap_grad(ctx.h, snaps.h, ne, W, _ptr(walkers), _ptr(out), _ptr(g), ctypes.byref(o),
                                       _stream()))
    return out, g


def force_bias(ctx: Context, L: torch.Tensor, walkers: torch.Tensor, ov: torch.Tensor, grad: torch.Tensor,
               sqrt_dt: float = 0.0):
    """xbar[W, nchol] = -sqrt_dt * i tr(L_gamma Phi g^T / O)  (sqrt_dt = 0: <v_gamma>)."""
    for t, nm in ((L, "L"), (walkers, "walkers"), (ov, "overlap"), (grad, "grad")):
        _need_cuda(t, nm, torch.complex128)
    W, n, ne = walkers.shape
    nchol = L.shape[0]
    xb = torch.empty((W, nchol), dtype=torch.complex128, device=walkers.device)
    ctx.check(ctx.lib.qcs_force_bias(ctx.h, n, ne, W, nchol, _ptr(L), _ptr(walkers), _ptr(ov), _ptr(grad),
                                     float(sqrt_dt), _ptr(xb), _stream()))
    return xb


def overlap_noalloc(Q: torch.Tensor, b: torch.Tensor, walkers: torch.Tensor, out: torch.Tensor,
                    status: torch.Tensor | None = None) -> None:
    """qcs_overlap_noalloc: overlaps into ``out`` (W complex128) with no device allocation by
    the library (its scratch is a fixed 32 MiB device array).  ``status`` is an optional
    int32 CUDA tensor of at least one element into which device status bits are OR-ed.
    Every tensor must live on the same device; the call runs there."""
    _need_cuda(Q, "Q", torch.float64)
    _need_cuda(b, "b", torch.uint8)
    _need_cuda(walkers, "walkers", torch.complex128)
    _need_cuda(out, "out", torch.complex128)
    if walkers.dim() != 3:
        raise ValueError("walkers must be (W, n, ne)")
    W, n, ne = walkers.shape
    if Q.dim() != 3 or Q.shape[1:] != (2 * n, 2 * n):
        raise ValueError(f"Q must be (P, {2 * n}, {2 * n}) for walkers with n = {n}")
    P = Q.shape[0]
    if tuple(b.shape) != (P, n):
        raise ValueError(f"b must be ({P}, {n})")
    if out.numel() < W:
        raise ValueError(f"out must hold at least {W} overlaps")
    if status is not None:
        _need_cuda(status, "status", torch.int32)
        if status.numel() < 1:
            raise ValueError("status must hold one int32")
    dev = walkers.device
    for t, nm in ((Q, "Q"), (b, "b"), (out, "out"), (status, "status")):
        if t is not None and t.device != dev:
            raise ValueError(f"{nm} lives on {t.device}, the walkers on {dev}")
    with torch.cuda.device(dev):
        rc = load().qcs_overlap_noalloc(n, ne, P, _ptr(Q), _ptr(b), W, _ptr(walkers), _ptr(out), _ptr(status),
                                        _stream())
    if rc != QCS_OK:
        why = ("the sizes need more than the fixed 32 MiB scratch, or invalid arguments" if rc == 1 else "")
        raise QCSError(rc, f"qcs_overlap_noalloc failed: {why}")


def flops_per_pair(n: int, ne: int, nodes: int = 0, flags: int = 0) -> float:
    return float(load().qcs_overlap_flops_per_pair(n, ne, nodes, flags))


def flops_breakdown(n: int, ne: int, nodes: int = 0, flags: int = 0) -> dict:
    """Host-only: the parts of flops_per_pair (congruence T, covariance B, Pfaffians)."""
    out = (ctypes.c_double * 3)()
    rc = load().qcs_overlap_flops_breakdown(n, ne, nodes, flags, out)
    if rc != QCS_OK:
        raise QCSError(rc, "qcs_overlap_flops_breakdown: sizes or nodes out of range")
    return {"T": out[0], "B": out[1], "pfaffian": out[2]}


def tc_work_per_pair(n: int, ne: int, nodes: int = 0, flags: int = 0) -> dict:
    """Host-only: FP64 flops and BF16 tensor-core flops per non-trivial pair when the
    congruence runs on tensor cores."""
    f, t = ctypes.c_double(), ctypes.c_double()
    rc = load().qcs_overlap_tc_work_per_pair(n, ne, nodes, flags, ctypes.byref(f), ctypes.byref(t))
    if rc != QCS_OK:
        raise QCSError(rc, "qcs_overlap_tc_work_per_pair: sizes or nodes out of range")
    return {"fp64": f.value, "tensor": t.value}


def grad_flops_per_pair(n: int, ne: int, nodes: int = 0, flags: int = 0) -> float:
    return float(load().qcs_grad_flops_per_pair(n, ne, nodes, flags))


def flops_per_pair_signed_perm(n: int, ne: int, nodes: int = 0, flags: int = 0) -> float:
    return float(load().qcs_overlap_flops_per_pair_signed_perm(n, ne, nodes, flags))


def grad_flops_per_pair_signed_perm(n: int, ne: int, nodes: int = 0, flags: int = 0) -> float:
    return float(load().qcs_grad_flops_per_pair_signed_perm(n, ne, nodes, flags))


def shadow_rdm(ctx: Context, snaps: Snapshots, R: torch.Tensor | None = None, deg4: bool = True):
    """Shadow estimates from the snapshot set (qcs_shadow_rdm): dict of device tensors
    gam2 (2n x 2n, <g~_mu g~_nu> = i gam2), gam4 (C(2n,4), when deg4), rdm1 (n x n
    complex) and npart (scalar)."""
    from math import comb

    n = snaps.n
    dev = f"cuda:{ctx.device}"
    if R is not None:
        _need_cuda(R, "R", torch.float64)
    gam2 = torch.empty((2 * n, 2 * n), dtype=torch.float64, device=dev)
    gam4 = torch.empty(comb(2 * n, 4), dtype=torch.float64, device=dev) if deg4 else None
    rdm1 = torch.empty((n, n), dtype=torch.complex128, device=dev)
    npart = torch.empty((), dtype=torch.float64, device=dev)
    ctx.check(ctx.lib.qcs_shadow_rdm(ctx.h, snaps.h, _ptr(R) if R is not None else None, _ptr(gam2),
                                     _ptr(gam4) if gam4 is not None else None, _ptr(rdm1), _ptr(npart), _stream()))
    return dict(gam2=gam2, gam4=gam4, rdm1=rdm1, npart=npart)


def vce_transform(ctx: Context, walkers: torch.Tensor, nc: int, na: int, nea: int, act: torch.Tensor | None = None,
                  row0: int = 0, col0: int = 0):
    """Virtual-correlation-energy transform of one spin sector (qcs_vce_transform).
    walkers: (W, NB, nc + nea) complex128.  The active walkers are written into act
    (W, R, C) complex128 at rows row0.. and columns col0.. (a new (W, na, nea) tensor
    when act is None); returns (act, factor[W])."""
    _need_cuda(walkers, "walkers", torch.complex128)
    W, NB, ne = walkers.shape
    if ne != nc + nea:
        raise ValueError("walkers must have nc + nea columns")
    if act is None:
        act = torch.zeros((W, na, nea), dtype=torch.complex128, device=walkers.device)
    _need_cuda(act, "act", torch.complex128)
    if act.shape[0] != W or row0 + na > act.shape[1] or col0 + nea > act.shape[2]:
        raise ValueError("act too small for the na x nea block at (row0, col0)")
    factor = torch.empty(W, dtype=torch.complex128, device=walkers.device)
    base = ctypes.c_void_p(act.data_ptr() + 16 * (row0 * act.shape[2] + col0)) if nea > 0 else None
    ctx.check(ctx.lib.qcs_vce_transform(ctx.h, NB, nc, na, nea, W, _ptr(walkers), base,
                                        act.shape[1] * act.shape[2], act.shape[2], _ptr(factor), _stream()))
    return act, factor


def local_energy(ctx: Context, snaps: Snapshots, walkers: torch.Tensor, L: torch.Tensor,
                 h: torch.Tensor | None = None, nodes: int = 0, flags: int = 0):
    """(overlap, e1, e2) per walker (qcs_local_energy): e1 = <Psi_T|hhat|phi>/O (None
    without h), e2 = sum_gamma <Psi_T|Lhat_gamma^2|phi>/O.  L: (nchol, n, n) complex128."""
    _need_cuda(walkers, "walkers", torch.complex128)
    _need_cuda(L, "L", torch.complex128)
    if h is not None:
        _need_cuda(h, "h", torch.complex128)
    W, n, ne = walkers.shape
    dev = walkers.device
    ov = torch.empty(W, dtype=torch.complex128, device=dev)
    e1 = torch.empty(W, dtype=torch.complex128, device=dev) if h is not None else None
    e2 = torch.empty(W, dtype=torch.complex128, device=dev)
    o = _opts(nodes, flags)
    ctx.check(ctx.lib.qcs_local_energy(ctx.h, snaps.h, ne, W, _ptr(walkers), L.shape[0], _ptr(L), _ptr(h),
                                       _ptr(ov), _ptr(e1), _ptr(e2), ctypes.byref(o), _stream()))
    return ov, e1, e2


def local_energy_flops_per_pair(n: int, ne: int, nchol: int, has_h: bool = True, nodes: int = 0,
                                flags: int = 0) -> float:
    return float(load().qcs_local_energy_flops_per_pair(n, ne, nchol, int(has_h), nodes, flags))


def shadow_rdm_flops(n: int, P: int) -> float:
    return float(load().qcs_shadow_rdm_flops(n, P))


def node_plan(n: int, ne: int, nodes: int = 0, flags: int = 0):
    """Host-only: (wnode, gamma) complex arrays of the node plan; the pair term
    is sum_k gamma_k pf(B + wnode_k D)."""
    import numpy as np

    nev = ctypes.c_int(0)
    w = (ctypes.c_double * (2 * MAX_NODES))()
    g = (ctypes.c_double * (2 * MAX_NODES))()
    rc = load().qcs_node_plan_get(n, ne, nodes, flags, ctypes.byref(nev), w, g)
    if rc != QCS_OK:
        raise QCSError(rc, "qcs_node_plan_get: sizes or nodes out of range")
    k = nev.value
    wn = np.array(w[: 2 * k]).view(np.complex128)
    gm = np.array(g[: 2 * k]).view(np.complex128)
    return wn, gm


class OverlapFn(torch.autograd.Function):
    """Differentiable shadow overlap.  Forward: qcs_overlap_grad (the gradient is
    computed alongside and kept); backward: PyTorch's convention for a
    holomorphic function, grad_walkers = conj(dO/dPhi) * grad_output."""

    @staticmethod
    def forward(ctx_, walkers, qctx, snaps):
        ov, g = overlap_grad(qctx, snaps, walkers.detach().contiguous())
        ctx_.save_for_backward(g)
        return ov

    @staticmethod
    def backward(ctx_, grad_out):
        (g,) = ctx_.saved_tensors
        return g.conj() * grad_out[:, None, None], None, None
