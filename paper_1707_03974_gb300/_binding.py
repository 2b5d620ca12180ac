"""ctypes binding of libparadeisos.so: argument marshalling only.

Every function here forwards to the C entry point of the same name declared in
include/paradeisos.h.  Device buffers are torch CUDA tensors (torch provides
memory and streams); all computation happens in the library's CUDA kernels.
If the library has not been built, every call raises: there is no CPU path.
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass
from typing import Optional, Sequence, Tuple

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "lib", "libparadeisos.so")

HB_F64, HB_F32, HB_FX64 = 0, 1, 2
STATUS = {0: "HB_OK", 1: "HB_ERR_INVALID_ARG", 2: "HB_ERR_OVERFLOW", 3: "HB_ERR_INVALID_STATE",
          4: "HB_ERR_OUT_OF_RANGE", 5: "HB_ERR_NO_MEMORY", 6: "HB_ERR_CUDA", 7: "HB_ERR_NOT_CONVERGED",
          8: "HB_ERR_TIMEOUT"}
STATUS_CODE = {v: k for k, v in STATUS.items()}

_lib = None


class HubbardError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        self.name = STATUS.get(status, f"HB_STATUS_{status}")
        super().__init__(f"{where}: {self.name}")


class HvConfig(ctypes.Structure):
    _fields_ = [("rows_per_cta", ctypes.c_int32), ("threads_per_cta", ctypes.c_int32),
                ("visit_order", ctypes.c_int32), ("ms", ctypes.c_float), ("split", ctypes.c_int32),
                ("up_block", ctypes.c_int32), ("up_threads", ctypes.c_int32), ("up_rows", ctypes.c_int32)]

    def as_dict(self):
        return {"rows_per_cta": self.rows_per_cta, "threads_per_cta": self.threads_per_cta,
                "visit_order": self.visit_order, "ms": self.ms, "split": self.split, "up_block": self.up_block,
                "up_threads": self.up_threads, "up_rows": self.up_rows}


class LanczosOpts(ctypes.Structure):
    _fields_ = [("maxit", ctypes.c_int32), ("reorth", ctypes.c_int32), ("vec_dtype", ctypes.c_int32),
                ("check_every", ctypes.c_int32), ("tol", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("fp64_finish", ctypes.c_int32), ("f32_tol_exp", ctypes.c_int32), ("store_basis", ctypes.c_int32)]


class LanczosInfo(ctypes.Structure):
    _fields_ = [("E0", ctypes.c_double), ("residual", ctypes.c_double), ("iterations", ctypes.c_int32),
                ("iterations_f32", ctypes.c_int32), ("status", ctypes.c_int32), ("converged", ctypes.c_int32),
                ("seconds", ctypes.c_double)]


class Ceilings(ctypes.Structure):
    _fields_ = [("sm_count", ctypes.c_int32), ("sm_clock_mhz", ctypes.c_double),
                ("fp64_fma_tflops", ctypes.c_double), ("fp32_fma_tflops", ctypes.c_double),
                ("int32_add_tops", ctypes.c_double), ("int64_add_tops", ctypes.c_double),
                ("smem_seq16_gbs", ctypes.c_double), ("smem_gather8_gbs", ctypes.c_double),
                ("smem_gather16_gbs", ctypes.c_double), ("smem_gather8_clk", ctypes.c_double),
                ("smem_gather16_clk", ctypes.c_double), ("l1_gbs", ctypes.c_double), ("l2_gbs", ctypes.c_double),
                ("hbm_read_gbs", ctypes.c_double), ("l2_window_bytes", ctypes.c_uint64),
                ("hbm_window_bytes", ctypes.c_uint64)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


def load():
    """Load libparadeisos.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"libparadeisos.so is not built ({LIB_PATH}); run __graft_entry__.build()")
    lib = ctypes.CDLL(LIB_PATH)
    P, U64, I32, D = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_double
    sig = {
        "hb_status_string": (ctypes.c_char_p, [ctypes.c_int]),
        "hubbard_basis_create": (ctypes.c_int, [I32, I32, P, P, D, I32, I32, ctypes.POINTER(P)]),
        "hubbard_basis_create_k": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.POINTER(ctypes.c_void_p)]),
        "hubbard_basis_destroy": (ctypes.c_int, [P]),
        "hubbard_basis_dim": (ctypes.c_int, [P, ctypes.POINTER(U64), ctypes.POINTER(U64), ctypes.POINTER(U64)]),
        "hubbard_set_U": (ctypes.c_int, [P, D]),
        "paradeisos_rank": (ctypes.c_int, [P, P, P, U64, P]),
        "paradeisos_unrank": (ctypes.c_int, [P, P, P, U64, P]),
        "hubbard_apply": (ctypes.c_int, [P, I32, P, P, P]),
        "hubbard_row_entries": (ctypes.c_int, [P, U64, ctypes.c_uint32, ctypes.c_uint32, P, P, P, P]),
        "hubbard_last_error": (ctypes.c_int, [P]),
        "lanczos_workspace_bytes": (ctypes.c_int, [P, ctypes.POINTER(LanczosOpts), ctypes.POINTER(U64)]),
        "lanczos_ground_state": (ctypes.c_int, [P, ctypes.POINTER(LanczosOpts), P, P, U64, P, P,
                                                ctypes.POINTER(D), ctypes.POINTER(LanczosInfo), P]),
        "hb_tridiag_lowest": (ctypes.c_int, [P, P, I32, ctypes.POINTER(D), ctypes.POINTER(D)]),
        "paradeisos_inv_create": (ctypes.c_int, [I32, I32, ctypes.POINTER(P)]),
        "lanczos_ritz_vector_f64": (ctypes.c_int, [P, ctypes.POINTER(LanczosOpts), P, P, U64, P, ctypes.POINTER(D),
                                                   ctypes.POINTER(LanczosInfo), P]),
        "hubbard_apply_c": (ctypes.c_int, [P, P, I32, I32, I32, I32, P, P, P, P]),
        "hb_continued_fraction": (ctypes.c_int, [P, P, I32, D, D, P, P, I32, P, P]),
        "paradeisos_inv_destroy": (ctypes.c_int, [P]),
        "paradeisos_inv_dim": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_uint64)]),
        "paradeisos_inv_rank": (ctypes.c_int, [P, P, P, ctypes.c_uint64, P]),
        "paradeisos_inv_unrank": (ctypes.c_int, [P, P, P, ctypes.c_uint64, P]),
        "paradeisos_inv_last_error": (ctypes.c_int, [P]),
        "hubbard_fixed_point_bits": (ctypes.c_int, [P, ctypes.POINTER(ctypes.c_int32)]),
        "lanczos_ritz_vector_f32": (ctypes.c_int, [P, ctypes.POINTER(LanczosOpts), P, P, U64, P,
                                                   ctypes.POINTER(D), ctypes.POINTER(LanczosInfo), P]),
        "mlp_create": (ctypes.c_int, [I32, U64, ctypes.POINTER(P)]),
        "mlp_destroy": (ctypes.c_int, [P]),
        "mlp_param_count": (ctypes.c_int, [P, ctypes.POINTER(U64)]),
        "mlp_get_params": (ctypes.c_int, [P, P]),
        "mlp_set_params": (ctypes.c_int, [P, P]),
        "mlp_forward": (ctypes.c_int, [P, P, U64, P, P]),
        "mlp_gradient": (ctypes.c_int, [P, P, U64, P, P, P, ctypes.c_float, P, P, P]),
        "mlp_adam_step": (ctypes.c_int, [P, ctypes.c_float, P]),
        "mlp_start_vector": (ctypes.c_int, [P, P, I32, P, P]),
        "mlp_last_error": (ctypes.c_int, [P]),
        "mlp_tc_gemm": (ctypes.c_int, [P, P, P, I32, I32, I32, P]),
        "mlp_activation": (ctypes.c_int, [P, U64, P, I32, P]),
        "mlp_sample_workspace_bytes": (ctypes.c_int, [P, U64, ctypes.POINTER(U64)]),
        "mlp_sample_training": (ctypes.c_int, [P, P, U64, U64, P, P, P, P, U64, P]),
        "hb_device_wait_selftest": (ctypes.c_int, [ctypes.c_uint32]),
        "hubbard_batch_create": (ctypes.c_int, [I32, P, ctypes.POINTER(P)]),
        "hubbard_batch_destroy": (ctypes.c_int, [P]),
        "hubbard_batch_layout": (ctypes.c_int, [P, P]),
        "hubbard_batch_apply": (ctypes.c_int, [P, I32, P, P, P]),
        "hubbard_batch_autotune": (ctypes.c_int, [P, I32, P, P, I32, ctypes.POINTER(HvConfig), P]),
        "hubbard_batch_get_config": (ctypes.c_int, [P, ctypes.POINTER(HvConfig)]),
        "hubbard_batch_set_config": (ctypes.c_int, [P, ctypes.POINTER(HvConfig)]),
        "lanczos_batch_workspace_bytes": (ctypes.c_int, [P, ctypes.POINTER(LanczosOpts), ctypes.POINTER(U64)]),
        "lanczos_batch_ground_state": (ctypes.c_int, [P, ctypes.POINTER(LanczosOpts), P, U64, P, P, P]),
        "lanczos_batch_wait_selftest": (ctypes.c_int, [P, ctypes.POINTER(LanczosOpts), P, U64, ctypes.c_int32,
                                                       ctypes.c_uint32, P]),
        "hubbard_get_hv_config": (ctypes.c_int, [P, I32, ctypes.POINTER(HvConfig)]),
        "hubbard_set_hv_config": (ctypes.c_int, [P, I32, ctypes.POINTER(HvConfig)]),
        "hubbard_autotune": (ctypes.c_int, [P, I32, P, P, I32, ctypes.POINTER(HvConfig), P]),
        "hubbard_convert": (ctypes.c_int, [P, I32, P, I32, P, U64, P]),
        "lanczos_step_scratch_bytes": (ctypes.c_int, [P, ctypes.POINTER(U64)]),
        "lanczos_step": (ctypes.c_int, [P, I32, P, P, P, P, P, P, P, U64, P, P, ctypes.POINTER(ctypes.c_uint32), P]),
        "lanczos_step_noalloc": (ctypes.c_int, [P, I32, P, P, P, P, P, P, P, P, ctypes.POINTER(ctypes.c_uint32), P]),
        "hb_measure_ceilings": (ctypes.c_int, [P, U64, ctypes.POINTER(Ceilings), P]),
        "hubbard_apply_timed": (ctypes.c_int, [P, I32, P, P, P, P, P, P]),
        "hb_host_alloc": (ctypes.c_int, [U64, ctypes.POINTER(P)]),
        "hb_host_free": (ctypes.c_int, [P]),
    }
    for name, (res, args) in sig.items():
        f = getattr(lib, name)
        f.restype = res
        f.argtypes = args
    _lib = lib
    return lib


def _check(status: int, where: str):
    if status != 0:
        raise HubbardError(status, where)


def _stream_ptr(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _ptr(t) -> ctypes.c_void_p:
    return ctypes.c_void_p(t.data_ptr()) if t is not None else ctypes.c_void_p(0)


# ---------------------------------------------------------------- handle + API

class Handle:
    """Owns one hb_handle (hubbard_basis_create / hubbard_basis_destroy)."""

    def __init__(self, L: int, bonds: Sequence[Tuple[int, int]], t: Sequence[float], U: float, N_up: int, N_dn: int):
        import numpy as np
        lib = load()
        b = np.ascontiguousarray(np.asarray(bonds, dtype=np.int32).reshape(-1, 2))
        tt = np.ascontiguousarray(np.asarray(t, dtype=np.float64).reshape(-1))
        if len(tt) != len(b):
            raise ValueError("bonds and t differ in length")
        h = ctypes.c_void_p()
        _check(lib.hubbard_basis_create(int(L), len(b), ctypes.c_void_p(b.ctypes.data), ctypes.c_void_p(tt.ctypes.data),
                                        float(U), int(N_up), int(N_dn), ctypes.byref(h)), "hubbard_basis_create")
        self._h = h
        self.L, self.N_up, self.N_dn, self.U = int(L), int(N_up), int(N_dn), float(U)
        self.n_bonds = len(b)
        D, Du, Dd = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(lib.hubbard_basis_dim(h, ctypes.byref(D), ctypes.byref(Du), ctypes.byref(Dd)), "hubbard_basis_dim")
        self.D, self.D_up, self.D_dn = D.value, Du.value, Dd.value

    @classmethod
    def momentum(cls, Lx: int, Ly: int, t: float, tp: float, U: float, N_up: int, N_dn: int, Kx: int, Ky: int):
        """Handle of one momentum sector (hubbard_basis_create_k): Lx x Ly periodic cluster (Ly = 1: ring),
        total momentum 2 pi (Kx/Lx, Ky/Ly)."""
        lib = load()
        self = cls.__new__(cls)
        h = ctypes.c_void_p()
        _check(lib.hubbard_basis_create_k(int(Lx), int(Ly), float(t), float(tp), float(U), int(N_up), int(N_dn),
                                          int(Kx), int(Ky), ctypes.byref(h)), "hubbard_basis_create_k")
        self._h = h
        self.L, self.N_up, self.N_dn, self.U = int(Lx * Ly), int(N_up), int(N_dn), float(U)
        self.n_bonds = 0
        self.Lx, self.Ly, self.K = int(Lx), int(Ly), (int(Kx), int(Ky))
        self.t, self.tp = float(t), float(tp)
        D, Du, Dd = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint64()
        _check(lib.hubbard_basis_dim(h, ctypes.byref(D), ctypes.byref(Du), ctypes.byref(Dd)), "hubbard_basis_dim")
        self.D, self.D_up, self.D_dn = D.value, Du.value, Dd.value
        return self

    @property
    def ptr(self):
        if self._h is None:
            raise RuntimeError("handle destroyed")
        return self._h

    def close(self):
        if getattr(self, "_h", None) is not None:
            load().hubbard_basis_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def hubbard_basis_create(L, bonds, t, U, N_up, N_dn) -> Handle:
    return Handle(L, bonds, t, U, N_up, N_dn)


def hubbard_basis_destroy(h: Handle):
    h.close()


def hubbard_set_U(h: Handle, U: float):
    _check(load().hubbard_set_U(h.ptr, float(U)), "hubbard_set_U")
    h.U = float(U)


def _need_cuda(*ts):
    for t in ts:
        if t is not None and not t.is_cuda:
            raise ValueError("device (CUDA) tensor required")
        if t is not None and not t.is_contiguous():
            raise ValueError("contiguous tensor required")


def paradeisos_rank(h: Handle, states, idx=None, stream=None):
    """Combined indices of combined strings (uint64 bit patterns held in int64 tensors)."""
    import torch
    _need_cuda(states)
    if idx is None:
        idx = torch.empty_like(states)
    _need_cuda(idx)
    _check(load().paradeisos_rank(h.ptr, _ptr(states), _ptr(idx), states.numel(), _stream_ptr(stream)), "paradeisos_rank")
    return idx


def paradeisos_unrank(h: Handle, idx, states=None, stream=None):
    import torch
    _need_cuda(idx)
    if states is None:
        states = torch.empty_like(idx)
    _need_cuda(states)
    _check(load().paradeisos_unrank(h.ptr, _ptr(idx), _ptr(states), idx.numel(), _stream_ptr(stream)), "paradeisos_unrank")
    return states


def _dtype_code(t):
    """float64 -> HB_F64, float32 -> HB_F32, int64 -> HB_FX64 (fixed point)."""
    import torch
    if t.dtype == torch.float64:
        return HB_F64
    if t.dtype == torch.float32:
        return HB_F32
    if t.dtype == torch.int64:
        return HB_FX64
    raise ValueError("vectors must be float64, float32 or int64 (fixed point)")


def hubbard_fixed_point_bits(h: "Handle") -> int:
    F = ctypes.c_int32()
    _check(load().hubbard_fixed_point_bits(h.ptr, ctypes.byref(F)), "hubbard_fixed_point_bits")
    return F.value


def hubbard_get_hv_config(h: "Handle", dtype) -> dict:
    c = HvConfig()
    _check(load().hubbard_get_hv_config(h.ptr, _dtype_of(dtype), ctypes.byref(c)), "hubbard_get_hv_config")
    return c.as_dict()


def hubbard_set_hv_config(h: "Handle", dtype, rows_per_cta=0, threads_per_cta=0, visit_order=1, split=0,
                          up_block=0, up_threads=0, up_rows=0, ms=None):
    c = HvConfig(int(rows_per_cta), int(threads_per_cta), int(visit_order), 0.0, int(split), int(up_block),
                 int(up_threads), int(up_rows))
    _check(load().hubbard_set_hv_config(h.ptr, _dtype_of(dtype), ctypes.byref(c)), "hubbard_set_hv_config")


def hubbard_autotune(h: "Handle", x, y, reps: int = 3, stream=None) -> dict:
    """Time every H·v launch configuration on x -> y, keep the fastest; returns it (with ms)."""
    _need_cuda(x, y)
    c = HvConfig()
    _check(load().hubbard_autotune(h.ptr, _dtype_code(x), _ptr(x), _ptr(y), int(reps), ctypes.byref(c),
                                   _stream_ptr(stream)), "hubbard_autotune")
    return c.as_dict()


def _dtype_of(dtype) -> int:
    import torch
    return {torch.float64: HB_F64, torch.float32: HB_F32, torch.int64: HB_FX64}[dtype] \
        if not isinstance(dtype, int) else dtype


def hubbard_convert(h: "Handle", x, out_dtype, stream=None):
    """float64 <-> fixed-point (int64) conversion of a device vector."""
    import torch
    _need_cuda(x)
    y = torch.empty(x.shape, dtype=out_dtype, device=x.device)
    _check(load().hubbard_convert(h.ptr, _dtype_code(x), _ptr(x), _dtype_code(y), _ptr(y), x.numel(),
                                  _stream_ptr(stream)), "hubbard_convert")
    return y


def hubbard_apply(h: Handle, x, y=None, stream=None):
    """y = H x (matrix-free)."""
    import torch
    _need_cuda(x)
    if x.numel() != h.D:
        raise ValueError(f"x has {x.numel()} elements, D = {h.D}")
    if y is None:
        y = torch.empty_like(x)
    _need_cuda(y)
    if y.dtype != x.dtype or y.numel() != h.D:
        raise ValueError("y must match x in dtype and size")
    _check(load().hubbard_apply(h.ptr, _dtype_code(x), _ptr(x), _ptr(y), _stream_ptr(stream)), "hubbard_apply")
    return y


def hubbard_apply_timed(h: Handle, x, y, ev_begin, ev_mid, ev_end, stream=None):
    """y = H x with CUDA events (torch.cuda.Event, timing enabled) recorded before the H·v, between its
    row pass and spin-up pass (split form; after the kernel otherwise) and at the end."""
    _need_cuda(x, y)
    if x.numel() != h.D or y.numel() != h.D or y.dtype != x.dtype:
        raise ValueError("x and y must have D elements of one dtype")
    evs = []
    for e in (ev_begin, ev_mid, ev_end):
        e.record()  # materialise the event; the library re-records it on the stream
        evs.append(ctypes.c_void_p(e.cuda_event))
    _check(load().hubbard_apply_timed(h.ptr, _dtype_code(x), _ptr(x), _ptr(y), *evs, _stream_ptr(stream)),
           "hubbard_apply_timed")
    return y


def hubbard_row_entries(h: Handle, row0: int, nrows: int, max_entries: Optional[int] = None, stream=None):
    import torch
    me = int(max_entries) if max_entries is not None else 1 + 2 * h.n_bonds
    dev = torch.device("cuda", torch.cuda.current_device())
    cols = torch.empty((nrows, me), dtype=torch.int64, device=dev)
    vals = torch.empty((nrows, me), dtype=torch.float64, device=dev)
    counts = torch.empty((nrows,), dtype=torch.int32, device=dev)
    _check(load().hubbard_row_entries(h.ptr, int(row0), int(nrows), me, _ptr(cols), _ptr(vals), _ptr(counts),
                                      _stream_ptr(stream)), "hubbard_row_entries")
    return cols, vals, counts


def hubbard_last_error(h: Handle) -> str:
    return STATUS[load().hubbard_last_error(h.ptr)]


@dataclass
class LanczosResult:
    E0: float
    residual: float
    iterations: int
    iterations_f32: int
    status: str
    converged: bool
    seconds: float
    alphas: list
    betas: list


def lanczos_ground_state(h: Handle, maxit: int = 300, tol: float = 1e-10, reorth: bool = False, dtype=None,
                         seed: int = 0, v0=None, check_every: int = 1, fp64_finish: bool = False,
                         f32_tol_exp: int = 0, store_basis: int = 0, workspace=None, stream=None,
                         raise_on_error: bool = True) -> LanczosResult:
    import torch
    dt = {None: HB_F64, torch.float64: HB_F64, torch.float32: HB_F32, torch.int64: HB_FX64}[dtype]
    fin = {False: 0, True: 1, "f64": 1, "fx64": 2}[fp64_finish] if not isinstance(fp64_finish, int) or \
        isinstance(fp64_finish, bool) else int(fp64_finish)
    o = LanczosOpts(int(maxit), int(bool(reorth)), dt, int(check_every), float(tol), int(seed) & ((1 << 64) - 1),
                    fin, int(f32_tol_exp), int(store_basis))
    lib = load()
    nb = ctypes.c_uint64()
    _check(lib.lanczos_workspace_bytes(h.ptr, ctypes.byref(o), ctypes.byref(nb)), "lanczos_workspace_bytes")
    dev = torch.device("cuda", torch.cuda.current_device())
    if workspace is None or workspace.numel() * workspace.element_size() < nb.value:
        workspace = torch.empty((max(1, nb.value),), dtype=torch.uint8, device=dev)
    if v0 is not None:
        _need_cuda(v0)
        if _dtype_code(v0) != dt or v0.numel() != h.D:
            raise ValueError("v0 must have the Krylov vector dtype and D elements")
    import numpy as np
    alphas = np.zeros(maxit + 1)
    betas = np.zeros(maxit + 1)
    E0 = ctypes.c_double(float("nan"))
    info = LanczosInfo()
    st = lib.lanczos_ground_state(h.ptr, ctypes.byref(o), _ptr(v0), _ptr(workspace),
                                  workspace.numel() * workspace.element_size(),
                                  ctypes.c_void_p(alphas.ctypes.data), ctypes.c_void_p(betas.ctypes.data),
                                  ctypes.byref(E0), ctypes.byref(info), _stream_ptr(stream))
    if st not in (0, 7) or (raise_on_error and st != 0):
        raise HubbardError(st, "lanczos_ground_state")
    n_last = info.iterations - info.iterations_f32 if (fp64_finish and info.iterations != info.iterations_f32) \
        else info.iterations
    return LanczosResult(E0.value, info.residual, info.iterations, info.iterations_f32, STATUS[st],
                         bool(info.converged), info.seconds, alphas[:n_last].tolist(), betas[:n_last].tolist())


def lanczos_step_scratch_bytes(h: Handle) -> int:
    n = ctypes.c_uint64()
    _check(load().lanczos_step_scratch_bytes(h.ptr, ctypes.byref(n)), "lanczos_step_scratch_bytes")
    return n.value


def lanczos_step(h: Handle, v, vprev, w, beta_prev, alpha, beta, scratch, ev_hv_begin=None, ev_hv_end=None,
                 launches: Optional[ctypes.c_uint32] = None, stream=None):
    """One three-term Lanczos step; alpha/beta/beta_prev are 1-element float64 CUDA tensors (or views)."""
    _need_cuda(v, w)
    code = _dtype_code(v)
    ev0 = ctypes.c_void_p(ev_hv_begin.cuda_event) if ev_hv_begin is not None else ctypes.c_void_p(0)
    ev1 = ctypes.c_void_p(ev_hv_end.cuda_event) if ev_hv_end is not None else ctypes.c_void_p(0)
    _check(load().lanczos_step(h.ptr, code, _ptr(v), _ptr(vprev), _ptr(w), _ptr(beta_prev), _ptr(alpha), _ptr(beta),
                               _ptr(scratch), scratch.numel() * scratch.element_size(), ev0, ev1,
                               ctypes.byref(launches) if launches is not None else None, _stream_ptr(stream)),
           "lanczos_step")


def lanczos_step_noalloc(h: Handle, v, vprev, w, beta_prev, alpha, beta, ev_hv_begin=None, ev_hv_end=None,
                         launches: Optional[ctypes.c_uint32] = None, stream=None):
    """lanczos_step with the reductions' scratch in the library's fixed device array (no allocation)."""
    _need_cuda(v, w)
    code = _dtype_code(v)
    ev0 = ctypes.c_void_p(ev_hv_begin.cuda_event) if ev_hv_begin is not None else ctypes.c_void_p(0)
    ev1 = ctypes.c_void_p(ev_hv_end.cuda_event) if ev_hv_end is not None else ctypes.c_void_p(0)
    _check(load().lanczos_step_noalloc(h.ptr, code, _ptr(v), _ptr(vprev), _ptr(w), _ptr(beta_prev), _ptr(alpha),
                                       _ptr(beta), ev0, ev1,
                                       ctypes.byref(launches) if launches is not None else None,
                                       _stream_ptr(stream)), "lanczos_step_noalloc")


def lanczos_ritz_vector_f32(h: Handle, maxit: int = 1000, tol: float = 1e-6, seed: int = 0, v0=None,
                            check_every: int = 1, stream=None):
    """(E0, normalised float32 ground-state vector, info dict) from float32 Lanczos + replay."""
    import torch
    o = LanczosOpts(int(maxit), 0, HB_F32, int(check_every), float(tol), int(seed) & ((1 << 64) - 1), 1, 0)
    lib = load()
    nb = ctypes.c_uint64()
    _check(lib.lanczos_workspace_bytes(h.ptr, ctypes.byref(o), ctypes.byref(nb)), "lanczos_workspace_bytes")
    dev = torch.device("cuda", torch.cuda.current_device())
    ws = torch.empty((nb.value,), dtype=torch.uint8, device=dev)
    ritz = torch.empty(h.D, dtype=torch.float32, device=dev)
    E0 = ctypes.c_double()
    info = LanczosInfo()
    st = lib.lanczos_ritz_vector_f32(h.ptr, ctypes.byref(o), _ptr(v0), _ptr(ws), nb.value, _ptr(ritz),
                                     ctypes.byref(E0), ctypes.byref(info), _stream_ptr(stream))
    if st not in (0, 7):
        raise HubbardError(st, "lanczos_ritz_vector_f32")
    return E0.value, ritz, {"iterations": info.iterations, "residual": info.residual, "converged": bool(info.converged)}


def hb_tridiag_lowest(alpha, beta):
    """Host utility of the library: lowest eigenvalue of a tridiagonal and its eigenvector's last entry."""
    import numpy as np
    a = np.ascontiguousarray(alpha, dtype=np.float64)
    b = np.ascontiguousarray(beta, dtype=np.float64)
    th, sl = ctypes.c_double(), ctypes.c_double()
    _check(load().hb_tridiag_lowest(ctypes.c_void_p(a.ctypes.data), ctypes.c_void_p(b.ctypes.data), len(a),
                                    ctypes.byref(th), ctypes.byref(sl)), "hb_tridiag_lowest")
    return th.value, sl.value


class Batch:
    """Owns an hb_batch_handle over a list of Handles (which must outlive it)."""

    def __init__(self, handles):
        import numpy as np
        lib = load()
        self.handles = list(handles)
        arr = (ctypes.c_void_p * len(self.handles))(*[h.ptr.value for h in self.handles])
        b = ctypes.c_void_p()
        _check(lib.hubbard_batch_create(len(self.handles), arr, ctypes.byref(b)), "hubbard_batch_create")
        self._b = b
        off = np.zeros(len(self.handles) + 1, dtype=np.uint64)
        _check(lib.hubbard_batch_layout(b, ctypes.c_void_p(off.ctypes.data)), "hubbard_batch_layout")
        self.offsets = off.astype(np.int64)
        self.total = int(off[-1])

    def close(self):
        if getattr(self, "_b", None) is not None:
            load().hubbard_batch_destroy(self._b)
            self._b = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def view(self, vec, k):
        """Instance k's part of a batch vector."""
        return vec[int(self.offsets[k]):int(self.offsets[k]) + self.handles[k].D]


def hubbard_batch_apply(b: Batch, x, y=None, stream=None):
    import torch
    _need_cuda(x)
    if x.numel() != b.total:
        raise ValueError("x must have the batch length")
    if y is None:
        y = torch.zeros_like(x)
    _check(load().hubbard_batch_apply(b._b, _dtype_code(x), _ptr(x), _ptr(y), _stream_ptr(stream)),
           "hubbard_batch_apply")
    return y


def hubbard_batch_get_config(b: Batch) -> dict:
    c = HvConfig()
    _check(load().hubbard_batch_get_config(b._b, ctypes.byref(c)), "hubbard_batch_get_config")
    return c.as_dict()


def hubbard_batch_set_config(b: Batch, rows_per_cta=0, threads_per_cta=0, split=0, up_block=0, up_threads=0,
                             up_rows=0):
    c = HvConfig(int(rows_per_cta), int(threads_per_cta), 1, 0.0, int(split), int(up_block), int(up_threads),
                 int(up_rows))
    _check(load().hubbard_batch_set_config(b._b, ctypes.byref(c)), "hubbard_batch_set_config")


def hubbard_batch_autotune(b: Batch, x, y, reps: int = 3, stream=None) -> dict:
    _need_cuda(x, y)
    c = HvConfig()
    _check(load().hubbard_batch_autotune(b._b, _dtype_code(x), _ptr(x), _ptr(y), int(reps), ctypes.byref(c),
                                         _stream_ptr(stream)), "hubbard_batch_autotune")
    return c.as_dict()


def lanczos_batch_ground_state(b: Batch, maxit: int = 1000, tol: float = 1e-10, dtype=None, seed: int = 0,
                               check_every: int = 10, workspace=None, stream=None):
    """Lowest eigenvalue of every instance; returns (E0 list, list of LanczosInfo dicts, status name)."""
    import numpy as np
    import torch
    dt = {None: HB_F64, torch.float64: HB_F64, torch.int64: HB_FX64}[dtype]
    o = LanczosOpts(int(maxit), 0, dt, int(check_every), float(tol), int(seed) & ((1 << 64) - 1), 0, 0)
    lib = load()
    nb = ctypes.c_uint64()
    _check(lib.lanczos_batch_workspace_bytes(b._b, ctypes.byref(o), ctypes.byref(nb)), "lanczos_batch_workspace_bytes")
    if workspace is None or workspace.numel() * workspace.element_size() < nb.value:
        workspace = torch.empty((nb.value,), dtype=torch.uint8, device=torch.device("cuda", torch.cuda.current_device()))
    n = len(b.handles)
    E0 = np.zeros(n)
    infos = (LanczosInfo * n)()
    st = lib.lanczos_batch_ground_state(b._b, ctypes.byref(o), _ptr(workspace),
                                        workspace.numel() * workspace.element_size(),
                                        ctypes.c_void_p(E0.ctypes.data), infos, _stream_ptr(stream))
    if st not in (0, 7):
        raise HubbardError(st, "lanczos_batch_ground_state")
    return E0.tolist(), [{"E0": i.E0, "residual": i.residual, "iterations": i.iterations,
                          "converged": bool(i.converged), "seconds": i.seconds} for i in infos], STATUS[st]


def lanczos_batch_wait_selftest(b: Batch, withhold_cta: int = 0, limit_ms: int = 50, dtype=None, stream=None) -> str:
    """One batched step with CTA `withhold_cta` never arriving at the first grid barrier: the other
    CTAs' bounded waits must give up (expected "HB_ERR_TIMEOUT")."""
    import torch
    dt = {None: HB_FX64, torch.float64: HB_F64, torch.int64: HB_FX64}[dtype]
    o = LanczosOpts(4, 0, dt, 1, 1e-10, 0, 0, 0)
    lib = load()
    nb = ctypes.c_uint64()
    _check(lib.lanczos_batch_workspace_bytes(b._b, ctypes.byref(o), ctypes.byref(nb)), "lanczos_batch_workspace_bytes")
    ws = torch.empty((nb.value,), dtype=torch.uint8, device=torch.device("cuda", torch.cuda.current_device()))
    return STATUS[lib.lanczos_batch_wait_selftest(b._b, ctypes.byref(o), _ptr(ws), nb.value, int(withhold_cta),
                                                  int(limit_ms), _stream_ptr(stream))]


# ---------------------------------------------------------------- learned start vector (paradeisos_mlp.h)

class Mlp:
    """Owns an hb_mlp_handle (mlp_create / mlp_destroy)."""

    def __init__(self, n_in: int, seed: int = 0):
        lib = load()
        m = ctypes.c_void_p()
        _check(lib.mlp_create(int(n_in), int(seed) & ((1 << 64) - 1), ctypes.byref(m)), "mlp_create")
        self._m = m
        self.n_in = int(n_in)
        P = ctypes.c_uint64()
        _check(lib.mlp_param_count(m, ctypes.byref(P)), "mlp_param_count")
        self.P = P.value

    @property
    def ptr(self):
        if self._m is None:
            raise RuntimeError("network destroyed")
        return self._m

    def close(self):
        if getattr(self, "_m", None) is not None:
            load().mlp_destroy(self._m)
            self._m = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def get_params(self):
        import numpy as np
        a = np.zeros(self.P, dtype=np.float32)
        _check(load().mlp_get_params(self.ptr, ctypes.c_void_p(a.ctypes.data)), "mlp_get_params")
        return a

    def set_params(self, a):
        import numpy as np
        a = np.ascontiguousarray(a, dtype=np.float32)
        if a.size != self.P:
            raise ValueError("parameter vector has the wrong length")
        _check(load().mlp_set_params(self.ptr, ctypes.c_void_p(a.ctypes.data)), "mlp_set_params")


def mlp_forward(m: Mlp, states, stream=None):
    import torch
    _need_cuda(states)
    out = torch.empty((states.numel(), 2), dtype=torch.float32, device=states.device)
    _check(load().mlp_forward(m.ptr, _ptr(states), states.numel(), _ptr(out), _stream_ptr(stream)), "mlp_forward")
    return out


def mlp_gradient(m: Mlp, states, t_log, t_sign, weights, lam: float = 1.0, stream=None):
    """Returns (grad tensor [P], loss tensor [1]); the gradient is also kept for mlp_adam_step."""
    import torch
    _need_cuda(states, t_log, t_sign, weights)
    g = torch.empty(m.P, dtype=torch.float32, device=states.device)
    loss = torch.empty(1, dtype=torch.float32, device=states.device)
    _check(load().mlp_gradient(m.ptr, _ptr(states), states.numel(), _ptr(t_log), _ptr(t_sign), _ptr(weights),
                               float(lam), _ptr(g), _ptr(loss), _stream_ptr(stream)), "mlp_gradient")
    return g, loss


def mlp_adam_step(m: Mlp, lr: float, stream=None):
    _check(load().mlp_adam_step(m.ptr, float(lr), _stream_ptr(stream)), "mlp_adam_step")


def mlp_start_vector(m: Mlp, h: Handle, dtype, stream=None):
    import torch
    v = torch.empty(h.D, dtype=dtype, device=torch.device("cuda", torch.cuda.current_device()))
    _check(load().mlp_start_vector(m.ptr, h.ptr, _dtype_code(v), _ptr(v), _stream_ptr(stream)), "mlp_start_vector")
    return v


def mlp_last_error(m: Mlp) -> str:
    return STATUS[load().mlp_last_error(m.ptr)]


def hb_device_wait_selftest(max_tries: int = 1000) -> str:
    return STATUS[load().hb_device_wait_selftest(int(max_tries))]


def mlp_sample_training(h: Handle, psi, n: int, seed: int = 0, stream=None):
    """(states int64, t_log float32, t_sign float32) of n basis states drawn with probability psi^2."""
    import torch
    _need_cuda(psi)
    if psi.dtype != torch.float32 or psi.numel() != h.D:
        raise ValueError("psi must be a float32 CUDA vector of D elements")
    lib = load()
    nb = ctypes.c_uint64()
    _check(lib.mlp_sample_workspace_bytes(h.ptr, int(n), ctypes.byref(nb)), "mlp_sample_workspace_bytes")
    ws = torch.empty((nb.value,), dtype=torch.uint8, device=psi.device)
    states = torch.empty(n, dtype=torch.int64, device=psi.device)
    t_log = torch.empty(n, dtype=torch.float32, device=psi.device)
    t_sign = torch.empty(n, dtype=torch.float32, device=psi.device)
    _check(lib.mlp_sample_training(h.ptr, _ptr(psi), int(n), int(seed) & ((1 << 64) - 1), _ptr(states), _ptr(t_log),
                                   _ptr(t_sign), _ptr(ws), nb.value, _stream_ptr(stream)), "mlp_sample_training")
    return states, t_log, t_sign


def mlp_activation(x, deriv: bool = False, stream=None):
    """gelu(x) or gelu'(x) of a float32 CUDA tensor, as the network's kernels evaluate it."""
    import torch
    _need_cuda(x)
    y = torch.empty_like(x)
    _check(load().mlp_activation(_ptr(x), x.numel(), _ptr(y), int(bool(deriv)), _stream_ptr(stream)), "mlp_activation")
    return y


def mlp_tc_gemm(A, B, stream=None):
    """C = A @ B^T on the library's tcgen05 kernel (A [M,K], B [N,K] bfloat16 CUDA tensors)."""
    import torch
    _need_cuda(A, B)
    M, K = A.shape
    N = B.shape[0]
    C = torch.empty((M, N), dtype=torch.float32, device=A.device)
    _check(load().mlp_tc_gemm(_ptr(A), _ptr(B), _ptr(C), int(M), int(N), int(K), _stream_ptr(stream)), "mlp_tc_gemm")
    return C


class Inversion:
    """Inversion-symmetric maps of n particles on an N-site chain (paradeisos_inv_*)."""

    def __init__(self, N: int, n: int):
        h = ctypes.c_void_p()
        _check(load().paradeisos_inv_create(int(N), int(n), ctypes.byref(h)), "paradeisos_inv_create")
        self._h, self.N, self.n = h, int(N), int(n)
        D = ctypes.c_uint64()
        _check(load().paradeisos_inv_dim(h, ctypes.byref(D)), "paradeisos_inv_dim")
        self.D = D.value

    def rank(self, states, stream=None):
        import torch
        _need_cuda(states)
        out = torch.empty_like(states)
        _check(load().paradeisos_inv_rank(self._h, _ptr(states), _ptr(out), states.numel(), _stream_ptr(stream)),
               "paradeisos_inv_rank")
        return out

    def unrank(self, idx, stream=None):
        import torch
        _need_cuda(idx)
        out = torch.empty_like(idx)
        _check(load().paradeisos_inv_unrank(self._h, _ptr(idx), _ptr(out), idx.numel(), _stream_ptr(stream)),
               "paradeisos_inv_unrank")
        return out

    def last_error(self) -> str:
        return STATUS[load().paradeisos_inv_last_error(self._h)]

    def close(self):
        if getattr(self, "_h", None) is not None:
            load().paradeisos_inv_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def lanczos_ritz_vector_f64(h: Handle, maxit: int = 3000, tol: float = 1e-10, seed: int = 0, v0=None,
                            check_every: int = 10, stream=None):
    """(E0, normalised float64 Ritz vector of E0, LanczosInfo) by float64 Lanczos and the replayed recurrence."""
    import torch
    lib = load()
    o = LanczosOpts(int(maxit), 0, HB_F64, int(check_every), float(tol), int(seed) & ((1 << 64) - 1), 0, 0)
    nb = ctypes.c_uint64()
    _check(lib.lanczos_workspace_bytes(h.ptr, ctypes.byref(o), ctypes.byref(nb)), "lanczos_workspace_bytes")
    dev = torch.device("cuda", torch.cuda.current_device())
    extra = (h.D * 8 + 255) // 256 * 256
    ws = torch.empty(nb.value + extra, dtype=torch.uint8, device=dev)
    ritz = torch.empty(h.D, dtype=torch.float64, device=dev)
    E0 = ctypes.c_double()
    info = LanczosInfo()
    st = lib.lanczos_ritz_vector_f64(h.ptr, ctypes.byref(o), _ptr(v0) if v0 is not None else None, _ptr(ws),
                                     ws.numel(), _ptr(ritz), ctypes.byref(E0), ctypes.byref(info),
                                     _stream_ptr(stream))
    if st not in (0, 7):  # HB_OK, HB_ERR_NOT_CONVERGED
        _check(st, "lanczos_ritz_vector_f64")
    return E0.value, ritz, info


def hubbard_apply_c(src: Handle, dst: Handle, op: str, spin: int, k: int, x, stream=None):
    """y = c_{k spin} x (op 'c') or c+_{k spin} x (op 'cdag') between momentum sectors; returns (y, ||y||^2)."""
    import torch
    _need_cuda(x)
    y = torch.empty(dst.D, dtype=x.dtype, device=x.device)
    n2 = torch.zeros(1, dtype=torch.float64, device=x.device)
    _check(load().hubbard_apply_c(src.ptr, dst.ptr, {"c": 0, "cdag": 1}[op], int(spin), int(k), _dtype_code(x),
                                  _ptr(x), _ptr(y), _ptr(n2), _stream_ptr(stream)), "hubbard_apply_c")
    return y, n2


def hb_continued_fraction(alphas, betas, norm2: float, E0: float, z):
    """G(z) of the Lanczos continued fraction at the complex points z (host utility)."""
    import numpy as np
    a = np.ascontiguousarray(np.asarray(alphas, dtype=np.float64))
    b = np.ascontiguousarray(np.asarray(betas, dtype=np.float64))
    z = np.asarray(z, dtype=complex).ravel()
    zr, zi = np.ascontiguousarray(z.real), np.ascontiguousarray(z.imag)
    gr, gi = np.empty(len(z)), np.empty(len(z))
    P = ctypes.c_void_p
    _check(load().hb_continued_fraction(P(a.ctypes.data), P(b.ctypes.data) if len(b) else None, len(a),
                                        float(norm2), float(E0), P(zr.ctypes.data), P(zi.ctypes.data), len(z),
                                        P(gr.ctypes.data), P(gi.ctypes.data)), "hb_continued_fraction")
    return gr + 1j * gi


def host_empty(n: int, dtype):
    """A pinned host tensor of n elements on huge pages (hb_host_alloc); the buffer is released
    (hb_host_free) when the tensor and all its views are gone."""
    import torch
    import weakref
    esize = torch.empty(0, dtype=dtype).element_size()
    nbytes = max(1, int(n)) * esize
    torch.cuda.init()  # torch's view of the context: is_pinned() and async copies see the registration
    lib = load()
    p = ctypes.c_void_p()
    _check(lib.hb_host_alloc(nbytes, ctypes.byref(p)), "hb_host_alloc")
    buf = (ctypes.c_char * nbytes).from_address(p.value)
    weakref.finalize(buf, lib.hb_host_free, ctypes.c_void_p(p.value))
    return torch.frombuffer(buf, dtype=dtype, count=int(n))


def hb_measure_ceilings(buffer, stream=None) -> dict:
    """Measured on-chip rates of the current device; buffer: a CUDA tensor of at least 64 MiB (overwritten)."""
    _need_cuda(buffer)
    c = Ceilings()
    _check(load().hb_measure_ceilings(_ptr(buffer), buffer.numel() * buffer.element_size(), ctypes.byref(c),
                                      _stream_ptr(stream)), "hb_measure_ceilings")
    return c.as_dict()
