"""Thin ctypes binding of libgh.so (include/gh.h).

Argument marshalling only: every step of the path runs in the library's CUDA
kernels. Functions named ``gh_*`` mirror the C entry points one to one;
``Context`` wraps them for convenience and allocates device buffers with
PyTorch (plumbing only). There is no fallback: if the library is missing the
first call raises.
"""
from __future__ import annotations

import ctypes
import os
import re

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "lib", "libgh.so")
HEADER = os.path.join(os.path.dirname(_HERE), "include", "gh.h")

GH_OK, GH_EINVAL, GH_ENOMEM, GH_ECUDA, GH_ETIMEOUT, GH_ENOTSUP = 0, -1, -2, -3, -4, -5
GH_TC_NOSWIZZLE, GH_TC_SW128 = 0, 1
GH_TC_SKIP_MMA = 1
GH_C64, GH_C16, GH_CBF16 = 0, 1, 2
GH_HOP, GH_EXACT, GH_INDIRECT = 0, 1, 2
(GH_K_RANGE_FFT, GH_K_DOPPLER_FFT, GH_K_COORD, GH_K_HOP_SCORE, GH_K_ARGMAX, GH_K_BOMP,
 GH_K_EXACT_S1, GH_K_EXACT_S2, GH_K_SYNTH, GH_K_POINTS, GH_K_DEFLATE) = range(11)
KERNEL_KINDS = {"range_fft": 0, "doppler_fft": 1, "coord": 2, "hop_score": 3, "argmax": 4,
                "bomp": 5, "exact_s1": 6, "exact_s2": 7, "synth": 8, "points": 9, "deflate": 10}


class GhRadar(ctypes.Structure):
    _fields_ = [("f0", ctypes.c_double), ("B", ctypes.c_double), ("Tc", ctypes.c_double),
                ("Ms", ctypes.c_int32), ("Mc", ctypes.c_int32), ("pad", ctypes.c_int32),
                ("reserved", ctypes.c_int32)]


class GhGrid(ctypes.Structure):
    _fields_ = [("lo", ctypes.c_double * 4), ("step", ctypes.c_double * 4), ("n", ctypes.c_int32 * 4)]


class GhFrame(ctypes.Structure):
    _fields_ = [("radar", GhRadar), ("tx", ctypes.c_double * 2), ("rx", ctypes.POINTER(ctypes.c_double)),
                ("Q", ctypes.c_int32), ("K", ctypes.c_int32), ("grid", GhGrid), ("Y", ctypes.c_void_p)]


class GhError(RuntimeError):
    def __init__(self, func, status, detail):
        super().__init__(f"{func} failed: {status} ({gh_status_str(status)}): {detail}")
        self.status = status


_lib = None
_P = ctypes.c_void_p
_I32 = ctypes.c_int32
_PD = ctypes.POINTER(ctypes.c_double)

_SIGNATURES = {
    "gh_create": (_I32, [ctypes.POINTER(_P), _I32, _P]),
    "gh_destroy": (None, [_P]),
    "gh_status_str": (ctypes.c_char_p, [_I32]),
    "gh_build_id": (ctypes.c_char_p, []),
    "gh_last_error": (ctypes.c_char_p, [_P]),
    "gh_make_maps": (_I32, [_P, ctypes.POINTER(GhRadar), _I32, _P, _P, _I32]),
    "gh_score_grid": (_I32, [_P, ctypes.POINTER(GhRadar), _P, _P, _I32, _P, _I32, ctypes.POINTER(GhGrid),
                             _P, _P, _P]),
    "gh_direct_exact": (_I32, [_P, ctypes.POINTER(GhRadar), _P, _P, _I32, _P, ctypes.POINTER(GhGrid), _P, _P, _P]),
    "gh_detect": (_I32, [_P, _I32, ctypes.POINTER(GhRadar), _P, _P, _I32, _P, ctypes.POINTER(GhGrid), _I32,
                         _P, _P, _P]),
    "gh_synth": (_I32, [_P, ctypes.POINTER(GhRadar), _P, _P, _I32, _I32, _P, _P, _P, _P]),
    "gh_coord_table": (_I32, [_P, ctypes.POINTER(GhRadar), _P, _P, _I32, ctypes.POINTER(GhGrid), _P, _P, _P, _P]),
    "gh_score_grid_noalloc": (_I32, [_P, ctypes.POINTER(GhRadar), _P, _P, _I32, _P, ctypes.POINTER(GhGrid),
                                     _P, _P, _P]),
    "gh_selftest_tcgen05": (_I32, [_P, _P, _P, _P, _I32, _I32]),
    "gh_selftest_tcgen05_ex": (_I32, [_P, _P, _P, _P, _I32, _I32, _I32, _I32, _I32]),
    "gh_probe_read_bandwidth": (_I32, [_P, ctypes.c_int64, _I32, _PD]),
    "gh_probe_smem_bandwidth": (_I32, [_P, _PD]),
    "gh_probe_issue_rate": (_I32, [_P, _PD]),
    "gh_set_timing": (_I32, [_P, _I32]),
    "gh_inject_fault": (_I32, [_P, _I32, _I32]),
    "gh_set_graphs": (_I32, [_P, _I32]),
    "gh_set_detect_maps": (_I32, [_P, _I32]),
    "gh_detect_batch": (_I32, [_P, _I32, _P, _P, _P, _P]),
    "gh_factorized": (_I32, [_P, _I32, ctypes.POINTER(GhRadar), _P, _P, _I32, _P, ctypes.POINTER(GhGrid), _P, _P,
                             _P]),
    "gh_set_batch_tuning": (_I32, [_P, _I32, _I32]),
    "gh_batch_tuning": (_I32, [_P, ctypes.POINTER(_I32), ctypes.POINTER(_I32)]),
    "gh_set_batch_tile": (_I32, [_P, _I32]),
    "gh_batch_tile": (_I32, [_P, ctypes.POINTER(_I32)]),
    "gh_batch_row_mode": (_I32, [_P, ctypes.POINTER(_I32)]),
    "gh_set_batch_row_mode": (_I32, [_P, _I32]),
    "gh_score_points": (_I32, [_P, ctypes.POINTER(GhRadar), _P, _P, _I32, _P, _I32, _P, ctypes.c_int64, _P]),
    "gh_score_points_adjoint": (_I32, [_P, ctypes.POINTER(GhRadar), _P, _P, _I32, _P, _I32, _P, ctypes.c_int64,
                                       _P, _P, _P, _P]),
    "gh_refine_points": (_I32, [_P, ctypes.POINTER(GhRadar), _P, _P, _I32, _P, _I32, _P, ctypes.c_int64, _I32,
                                ctypes.c_double, ctypes.c_double, ctypes.c_double, _P]),
    "gh_kernel_stats": (_I32, [_P, _I32, _PD, ctypes.POINTER(ctypes.c_int64)]),
    "gh_reset_stats": (_I32, [_P]),
    "gh_launch_count": (ctypes.c_int64, [_P]),
}


def load(path: str = LIB_PATH):
    """Load libgh.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"libgh.so not found at {path}: build it with "
                           "`python -m paper_2307_16550_gb300.build` (there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def header_functions(path: str = HEADER):
    """Names of the entry points include/gh.h declares."""
    text = open(path).read()
    return re.findall(r"^GH_API\s+[\w\s\*]+?\b(gh_\w+)\s*\(", text, flags=re.M)


def gh_status_str(status: int) -> str:
    return load().gh_status_str(status).decode()


def gh_build_id() -> str:
    """Build id compiled into the loaded library (see include/gh.h)."""
    return load().gh_build_id().decode()


def _ptr(x):
    """Raw address of a torch tensor, numpy array or None."""
    if x is None:
        return None
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return ctypes.c_void_p(x.data_ptr())
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return ctypes.c_void_p(x.ctypes.data)
    if isinstance(x, int):
        return ctypes.c_void_p(x)
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def radar_struct(radar) -> GhRadar:
    return GhRadar(float(radar.f0), float(radar.B), float(radar.Tc), int(radar.Ms), int(radar.Mc),
                   int(getattr(radar, "pad", 4)), 0)


def grid_struct(grid) -> GhGrid:
    g = GhGrid()
    for a in range(4):
        g.lo[a] = float(grid.lo[a])
        g.step[a] = float(grid.step[a])
        g.n[a] = int(grid.n[a])
    return g


def _f64(a, shape=None):
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    if shape is not None:
        arr = arr.reshape(shape)
    return arr


def gh_score_grid_noalloc(stream, radar, tx, rx, Q, maps, grid, scores=None):
    """Allocation-free hopping score and argmax (see include/gh.h); runs on
    `stream` (a torch.cuda.Stream, a raw cudaStream_t or None for the legacy
    default stream) on the current device. Returns (cell, score)."""
    lib = load()
    txa, rxa = _f64(tx, (2,)), _f64(rx, (-1,))
    cell = ctypes.c_int64(-1)
    score = ctypes.c_float(0.0)
    h = None if stream is None else ctypes.c_void_p(int(getattr(stream, "cuda_stream", stream)) or None)
    st = lib.gh_score_grid_noalloc(h, ctypes.byref(radar_struct(radar)), _ptr(txa), _ptr(rxa), int(Q), _ptr(maps),
                                   ctypes.byref(grid_struct(grid)), _ptr(scores), ctypes.byref(cell),
                                   ctypes.byref(score))
    if st != GH_OK:
        raise GhError("gh_score_grid_noalloc", st, "no context: see the status code")
    return cell.value, score.value


class Context:
    """A libgh context on one CUDA device (owns the library workspace)."""

    def __init__(self, device: int = 0, stream="torch"):
        """stream: "torch" (default) runs on PyTorch's current stream of the
        device, so results are ordered with torch ops; None lets the library
        create its own stream; or a torch.cuda.Stream / raw cudaStream_t."""
        lib = load()
        self._lib = lib
        h = ctypes.c_void_p()
        if isinstance(stream, str) and stream == "torch":
            import torch
            stream = torch.cuda.current_stream(device).cuda_stream
        if stream is None:
            s = None
        else:
            handle = int(getattr(stream, "cuda_stream", stream))
            s = ctypes.c_void_p(handle if handle != 0 else 1)  # 0x1: cudaStreamLegacy
        st = lib.gh_create(ctypes.byref(h), int(device), s)
        if st != GH_OK:
            raise GhError("gh_create", st, "")
        self.handle = h
        self.device = int(device)

    def close(self):
        if getattr(self, "handle", None) is not None and self.handle.value:
            self._lib.gh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _check(self, name, st):
        if st != GH_OK:
            raise GhError(name, st, self._lib.gh_last_error(self.handle).decode())

    # -- entry points -----------------------------------------------------
    def gh_make_maps(self, radar, Q, Y, maps, map_dtype=GH_C64):
        self._check("gh_make_maps", self._lib.gh_make_maps(self.handle, ctypes.byref(radar_struct(radar)), int(Q),
                                                           _ptr(Y), _ptr(maps), int(map_dtype)))

    def gh_score_grid(self, radar, tx, rx, Q, maps, grid, scores=None, map_dtype=GH_C64):
        txa, rxa = _f64(tx, (2,)), _f64(rx, (-1,))
        cell = ctypes.c_int64(-1)
        score = ctypes.c_float(0.0)
        self._check("gh_score_grid", self._lib.gh_score_grid(
            self.handle, ctypes.byref(radar_struct(radar)), _ptr(txa), _ptr(rxa), int(Q), _ptr(maps),
            int(map_dtype), ctypes.byref(grid_struct(grid)), _ptr(scores), ctypes.byref(cell), ctypes.byref(score)))
        return cell.value, score.value

    def gh_direct_exact(self, radar, tx, rx, Q, Y, grid, scores=None):
        txa, rxa = _f64(tx, (2,)), _f64(rx, (-1,))
        cell = ctypes.c_int64(-1)
        score = ctypes.c_float(0.0)
        self._check("gh_direct_exact", self._lib.gh_direct_exact(
            self.handle, ctypes.byref(radar_struct(radar)), _ptr(txa), _ptr(rxa), int(Q), _ptr(Y),
            ctypes.byref(grid_struct(grid)), _ptr(scores), ctypes.byref(cell), ctypes.byref(score)))
        return cell.value, score.value

    def gh_detect(self, method, radar, tx, rx, Q, Y, grid, K):
        txa, rxa = _f64(tx, (2,)), _f64(rx, (-1,))
        cells = np.zeros(K, np.int64)
        scores = np.zeros(K, np.float32)
        alpha = np.zeros((K, Q, 2), np.float64)
        self._check("gh_detect", self._lib.gh_detect(
            self.handle, int(method), ctypes.byref(radar_struct(radar)), _ptr(txa), _ptr(rxa), int(Q), _ptr(Y),
            ctypes.byref(grid_struct(grid)), int(K), _ptr(cells), _ptr(scores), _ptr(alpha)))
        return cells, scores, alpha[..., 0] + 1j * alpha[..., 1]

    def gh_synth(self, radar, tx, rx, Q, targets, alpha, noise, Y):
        txa, rxa = _f64(tx, (2,)), _f64(rx, (-1,))
        tg = _f64(targets, (-1, 4))
        T = tg.shape[0]
        al = np.ascontiguousarray(np.stack([np.real(alpha), np.imag(alpha)], axis=-1).astype(np.float64))
        self._check("gh_synth", self._lib.gh_synth(
            self.handle, ctypes.byref(radar_struct(radar)), _ptr(txa), _ptr(rxa), int(Q), int(T),
            _ptr(tg) if T else None, _ptr(al) if T else None, _ptr(noise), _ptr(Y)))

    def gh_coord_table(self, radar, tx, rx, Q, grid):
        txa, rxa = _f64(tx, (2,)), _f64(rx, (-1,))
        nx, ny = int(grid.n[0]), int(grid.n[1])
        ib = np.zeros((nx, ny, Q), np.int32)
        tau = np.zeros((nx, ny, Q), np.float64)
        coef = np.zeros((nx, ny, Q, 3), np.float32)
        w = np.zeros((nx, ny, Q, 2), np.float64)
        self._check("gh_coord_table", self._lib.gh_coord_table(
            self.handle, ctypes.byref(radar_struct(radar)), _ptr(txa), _ptr(rxa), int(Q),
            ctypes.byref(grid_struct(grid)), _ptr(ib), _ptr(tau), _ptr(coef), _ptr(w)))
        return ib, tau, coef, w

    def gh_selftest_tcgen05(self, A, B):
        """D = A @ B.T on the tensor cores (A: 128 x K, B: N x K, rounded to BF16)."""
        A = np.ascontiguousarray(A, dtype=np.float32)
        B = np.ascontiguousarray(B, dtype=np.float32)
        N, K = B.shape
        D = np.zeros((128, N), np.float32)
        self._check("gh_selftest_tcgen05", self._lib.gh_selftest_tcgen05(self.handle, _ptr(A), _ptr(B), _ptr(D),
                                                                         int(N), int(K)))
        return D

    def gh_selftest_tcgen05_ex(self, A, B, layout=GH_TC_NOSWIZZLE, flags=0, wait_polls=0):
        """As gh_selftest_tcgen05, with the operand layout, flags and wait limit
        of include/gh.h."""
        A = np.ascontiguousarray(A, dtype=np.float32)
        B = np.ascontiguousarray(B, dtype=np.float32)
        N, K = B.shape
        D = np.zeros((128, N), np.float32)
        self._check("gh_selftest_tcgen05_ex", self._lib.gh_selftest_tcgen05_ex(
            self.handle, _ptr(A), _ptr(B), _ptr(D), int(N), int(K), int(layout), int(flags), int(wait_polls)))
        return D

    def gh_probe_read_bandwidth(self, nbytes, reps=20):
        """Read bandwidth in GB/s over a device buffer of nbytes (L2 if small, DRAM if large)."""
        g = ctypes.c_double(0)
        self._check("gh_probe_read_bandwidth",
                    self._lib.gh_probe_read_bandwidth(self.handle, int(nbytes), int(reps), ctypes.byref(g)))
        return g.value

    def gh_probe_smem_bandwidth(self):
        """Shared-memory load bandwidth of the GPU, GB/s."""
        v = ctypes.c_double(0.0)
        self._check("gh_probe_smem_bandwidth", self._lib.gh_probe_smem_bandwidth(self.handle, ctypes.byref(v)))
        return v.value

    def gh_probe_issue_rate(self):
        """Warp instructions per second the GPU issues (independent FP32 FMAs)."""
        v = ctypes.c_double(0.0)
        self._check("gh_probe_issue_rate", self._lib.gh_probe_issue_rate(self.handle, ctypes.byref(v)))
        return v.value

    def gh_set_timing(self, enable):
        """True: time every kernel class; False: none; a kind name, an int mask
        or an iterable of kind names: only those classes."""
        if enable is True:
            mask = -1
        elif enable is False or enable is None:
            mask = 0
        elif isinstance(enable, str):
            mask = 1 << KERNEL_KINDS[enable]
        elif isinstance(enable, int):
            mask = enable
        else:
            mask = 0
            for k in enable:
                mask |= 1 << KERNEL_KINDS[k]
        self._check("gh_set_timing", self._lib.gh_set_timing(self.handle, int(mask)))

    def gh_score_points(self, radar, tx, rx_dev, Q, maps, points, P, scores, map_dtype=GH_C64):
        txa = _f64(tx, (2,))
        self._check("gh_score_points", self._lib.gh_score_points(
            self.handle, ctypes.byref(radar_struct(radar)), _ptr(txa), _ptr(rx_dev), int(Q), _ptr(maps),
            int(map_dtype), _ptr(points), int(P), _ptr(scores)))

    def gh_score_points_adjoint(self, radar, tx, rx_dev, Q, maps, points, P, dscores, dpoints=None, drx=None,
                                dmaps=None, map_dtype=GH_C64):
        txa = _f64(tx, (2,))
        self._check("gh_score_points_adjoint", self._lib.gh_score_points_adjoint(
            self.handle, ctypes.byref(radar_struct(radar)), _ptr(txa), _ptr(rx_dev), int(Q), _ptr(maps),
            int(map_dtype), _ptr(points), int(P), _ptr(dscores), _ptr(dpoints), _ptr(drx), _ptr(dmaps)))

    def gh_refine_points(self, radar, tx, rx_dev, Q, maps, points, P, iters, scale_xy, scale_v, step=1.0,
                         scores=None, map_dtype=GH_C64):
        txa = _f64(tx, (2,))
        self._check("gh_refine_points", self._lib.gh_refine_points(
            self.handle, ctypes.byref(radar_struct(radar)), _ptr(txa), _ptr(rx_dev), int(Q), _ptr(maps),
            int(map_dtype), _ptr(points), int(P), int(iters), float(scale_xy), float(scale_v), float(step),
            _ptr(scores)))

    def gh_detect_batch(self, frames):
        """frames: list of (radar, tx, rx, Q, Y_dev, grid, K). Returns per frame
        (cells int64[K], scores float32[K], alpha complex128[K][Q])."""
        n = len(frames)
        arr = (GhFrame * n)()
        keep = []
        total_k = sum(int(f[6]) for f in frames)
        total_a = sum(int(f[6]) * int(f[3]) for f in frames)
        for i, (radar, tx, rx, Q, Y, grid, K) in enumerate(frames):
            rxa = _f64(rx, (-1,))
            keep.append(rxa)
            fr = arr[i]
            fr.radar = radar_struct(radar)
            fr.tx[0], fr.tx[1] = float(tx[0]), float(tx[1])
            fr.rx = rxa.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
            fr.Q = int(Q)
            fr.K = int(K)
            fr.grid = grid_struct(grid)
            fr.Y = _ptr(Y)
        cells = np.zeros(total_k, np.int64)
        scores = np.zeros(total_k, np.float32)
        alpha = np.zeros((total_a, 2), np.float64)
        self._check("gh_detect_batch", self._lib.gh_detect_batch(self.handle, n, ctypes.cast(arr, _P), _ptr(cells),
                                                                 _ptr(scores), _ptr(alpha)))
        out, oc, oa = [], 0, 0
        for (_, _, _, Q, _, _, K) in frames:
            a = alpha[oa:oa + K * Q]
            out.append((cells[oc:oc + K], scores[oc:oc + K], (a[:, 0] + 1j * a[:, 1]).reshape(K, Q)))
            oc += K
            oa += K * Q
        return out

    def gh_factorized(self, method, radar, tx, rx, Q, Y, grid, loc_scores=None):
        """The paper's factorised estimators (GH_HOP, GH_EXACT) or the indirect
        method (GH_INDIRECT): (4D cell, (location value, velocity value))."""
        txa, rxa = _f64(tx, (2,)), _f64(rx, (-1,))
        cell = np.zeros(1, np.int64)
        vals = np.zeros(2, np.float64)
        self._check("gh_factorized", self._lib.gh_factorized(
            self.handle, int(method), ctypes.byref(radar_struct(radar)), _ptr(txa), _ptr(rxa), int(Q), _ptr(Y),
            ctypes.byref(grid_struct(grid)), _ptr(cell), _ptr(vals), _ptr(loc_scores)))
        return int(cell[0]), (float(vals[0]), float(vals[1]))

    def gh_set_batch_tuning(self, cells_per_lane=0, warps=0):
        self._check("gh_set_batch_tuning", self._lib.gh_set_batch_tuning(self.handle, int(cells_per_lane), int(warps)))

    def gh_batch_tuning(self):
        a, w = _I32(0), _I32(0)
        self._check("gh_batch_tuning", self._lib.gh_batch_tuning(self.handle, ctypes.byref(a), ctypes.byref(w)))
        return a.value, w.value

    def gh_set_batch_tile(self, cells_per_item=0):
        self._check("gh_set_batch_tile", self._lib.gh_set_batch_tile(self.handle, int(cells_per_item)))

    def gh_batch_row_mode(self):
        """1: the heaviest scorer group built one receiver's power row at a time; 0: all at once;
        2: all at once, shared by two warps per (x, y) cell."""
        m = _I32(0)
        self._check("gh_batch_row_mode", self._lib.gh_batch_row_mode(self.handle, ctypes.byref(m)))
        return m.value

    def gh_set_batch_row_mode(self, row_mode=-1):
        self._check("gh_set_batch_row_mode", self._lib.gh_set_batch_row_mode(self.handle, int(row_mode)))

    def gh_batch_tile(self):
        t = _I32(0)
        self._check("gh_batch_tile", self._lib.gh_batch_tile(self.handle, ctypes.byref(t)))
        return t.value

    def gh_set_detect_maps(self, map_dtype):
        """Storage type of the maps gh_detect makes for GH_HOP (GH_C64, GH_C16, GH_CBF16)."""
        self._check("gh_set_detect_maps", self._lib.gh_set_detect_maps(self.handle, int(map_dtype)))

    def gh_inject_fault(self, status, after=0):
        """Arms one host-side fault (see include/gh.h); GH_OK disarms."""
        self._check("gh_inject_fault", self._lib.gh_inject_fault(self.handle, int(status), int(after)))

    def gh_set_graphs(self, enable: bool):
        self._check("gh_set_graphs", self._lib.gh_set_graphs(self.handle, int(bool(enable))))

    def gh_kernel_stats(self, kind):
        ms = ctypes.c_double(0)
        n = ctypes.c_int64(0)
        k = KERNEL_KINDS[kind] if isinstance(kind, str) else int(kind)
        self._check("gh_kernel_stats", self._lib.gh_kernel_stats(self.handle, k, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def gh_reset_stats(self):
        self._check("gh_reset_stats", self._lib.gh_reset_stats(self.handle))

    def gh_launch_count(self) -> int:
        return int(self._lib.gh_launch_count(self.handle))

    # -- conveniences (allocate outputs with torch) -------------------------
    def _torch(self):
        import torch
        return torch

    def maps(self, radar, Y, map_dtype=GH_C64):
        """Range-Doppler maps of a device measurement Y (complex64 [Q][Mc][Ms]):
        complex64 [Q][Nr][Nd] for GH_C64, float16 / bfloat16 [Q][Nr][Nd][2]
        (2^-s times the values, s = log2(Ms Mc)) for GH_C16 / GH_CBF16."""
        torch = self._torch()
        Q = Y.shape[0]
        shape = (Q, radar.pad * radar.Ms, radar.pad * radar.Mc)
        if map_dtype == GH_C64:
            out = torch.empty(shape, dtype=torch.complex64, device=Y.device)
        else:
            dt = torch.float16 if map_dtype == GH_C16 else torch.bfloat16
            out = torch.empty(shape + (2,), dtype=dt, device=Y.device)
        self.gh_make_maps(radar, Q, Y, out, map_dtype)
        return out

    @staticmethod
    def map_dtype_of(maps):
        import torch
        return {torch.complex64: GH_C64, torch.float16: GH_C16, torch.bfloat16: GH_CBF16}[maps.dtype]

    def scores(self, radar, tx, rx, maps, grid):
        """Hopping scores of every cell (float32 [nx][ny][nvx][nvy]) and the argmax."""
        torch = self._torch()
        out = torch.empty(tuple(int(v) for v in grid.n), dtype=torch.float32, device=maps.device)
        cell, score = self.gh_score_grid(radar, tx, rx, maps.shape[0], maps, grid, out,
                                         map_dtype=self.map_dtype_of(maps))
        return out, cell, score

    def exact_scores(self, radar, tx, rx, Y, grid):
        torch = self._torch()
        out = torch.empty(tuple(int(v) for v in grid.n), dtype=torch.float32, device="cuda:%d" % self.device)
        cell, score = self.gh_direct_exact(radar, tx, rx, Y.shape[0], Y, grid, out)
        return out, cell, score

    def synth(self, radar, tx, rx, targets, alpha, noise=None):
        """Measurement of the signal model on the device (complex64 [Q][Mc][Ms])."""
        torch = self._torch()
        Q = np.asarray(rx).reshape(-1, 2).shape[0]
        Y = torch.empty((Q, radar.Mc, radar.Ms), dtype=torch.complex64, device="cuda:%d" % self.device)
        self.gh_synth(radar, tx, rx, Q, targets, alpha, noise, Y)
        return Y
