"""ctypes binding of ``libtmcs.so`` (argument marshalling only).

Function names mirror the C ABI in ``include/tmcs.h``; every sampling step
runs in the library's CUDA kernels. Device buffers are PyTorch CUDA tensors
(int64 or uint64, contiguous; their bits are the detector words) or raw
device pointers; streams are ``torch.cuda.Stream`` objects, raw
``cudaStream_t`` integers, or None for the current PyTorch stream.

The library must be built (``python -m paper_2504_05611_gb300.build`` or
``__graft_entry__.build()``); importing this module does not build it, and
every call raises ``RuntimeError`` if it is missing. There is no CPU path.
"""
from __future__ import annotations

import ctypes
import os
from typing import Dict, Iterable, List, Optional, Sequence, Tuple

import numpy as np

from .circuits import OPCODE_ID, Circuit

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libtmcs.so")

TMCS_OK = 0
STATUS = {0: "TMCS_OK", 1: "TMCS_E_INVALID", 2: "TMCS_E_NONDETERMINISTIC", 3: "TMCS_E_OOM",
          4: "TMCS_E_CUDA", 5: "TMCS_E_TIMEOUT", 6: "TMCS_E_BUFFER"}
TMCS_FLAG_NO_AUDIT = 0x1
TMCS_FLAG_NO_PRUNE = 0x2

OP_DTYPE = np.dtype([("code", "<u4"), ("n_targets", "<u4"), ("p", "<f8"), ("arg", "<u4"),
                     ("arg2", "<u4"), ("targets", "<u8")])
assert OP_DTYPE.itemsize == 32

STATS_FIELDS = ("n_layers", "n_slots", "n_xor", "n_zero", "n_copy", "n_noise_ops", "n_noise_units",
                "n_noise_segments", "n_parity_terms", "live_components", "pruned_updates",
                "sig_ok", "sig_window", "sig_steps", "sig_items", "sig_generators", "sig_entries",
                "sig_build_us", "sig_max_step_items", "sig_schedules", "sig_min_window", "sig_pipe_schedules")


class TmcsError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class _Job(ctypes.Structure):
    _fields_ = [("c", ctypes.c_void_p), ("shots", ctypes.c_uint64), ("seed", ctypes.c_uint64),
                ("det", ctypes.c_void_p), ("obs", ctypes.c_void_p)]


class _Stats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_uint64) for f in STATS_FIELDS]


class _ServerConfig(ctypes.Structure):
    _fields_ = [("n_streams", ctypes.c_uint32), ("slice_chunks", ctypes.c_uint32), ("arena_bytes", ctypes.c_uint64)]


SERVER_STATS_FIELDS = (("submitted", ctypes.c_uint64), ("completed", ctypes.c_uint64), ("failed", ctypes.c_uint64),
                       ("queued", ctypes.c_uint64), ("running", ctypes.c_uint64), ("arena_bytes", ctypes.c_uint64),
                       ("arena_in_use", ctypes.c_uint64), ("latency_p50_s", ctypes.c_double),
                       ("latency_p99_s", ctypes.c_double), ("latency_mean_s", ctypes.c_double),
                       ("busy_seconds", ctypes.c_double), ("shots_done", ctypes.c_uint64))


class _ServerStats(ctypes.Structure):
    _fields_ = list(SERVER_STATS_FIELDS)


REQ_STATES = {0: "queued", 1: "running", 2: "done", 3: "failed"}


_lib: Optional[ctypes.CDLL] = None


def lib() -> ctypes.CDLL:
    """Load libtmcs.so (once); raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2504_05611_gb300.build` (needs nvcc)")
        L = ctypes.CDLL(LIB_PATH)
        P, U64, I = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int
        L.tmcs_circuit_build.argtypes = [P, ctypes.c_size_t, ctypes.c_uint32, ctypes.POINTER(P)]
        L.tmcs_circuit_free.argtypes = [P]
        L.tmcs_circuit_info.argtypes = [P, P, P, P, P, P]
        L.tmcs_circuit_stats.argtypes = [P, P]
        L.tmcs_reference_sample.argtypes = [P, P]
        L.tmcs_sample.argtypes = [P, U64, U64, P, P, P]
        L.tmcs_sample_range.argtypes = [P, U64, U64, U64, P, P, P]
        L.tmcs_batch_sample.argtypes = [P, ctypes.c_size_t, P]
        L.tmcs_debug_gap_table.argtypes = [ctypes.c_double, P]
        L.tmcs_debug_gap_counts.argtypes = [ctypes.c_double, P, U64, P, I, P]
        L.tmcs_sample_noalloc.argtypes = [P, U64, U64, U64, P, P, P]
        L.tmcs_check_device.argtypes = []
        L.tmcs_fault_count.argtypes = [P, ctypes.POINTER(ctypes.c_uint64)]
        L.tmcs_fault_signatures.argtypes = [P, U64, U64, P, P, P]
        L.tmcs_sample_measurements.argtypes = [P, U64, U64, U64, P, P]
        L.tmcs_fault_outputs.argtypes = [P, U64, P, ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint32)]
        L.tmcs_dem_columns.argtypes = [P, ctypes.POINTER(U64), ctypes.POINTER(U64), P, P, P, P]
        L.tmcs_launch_shape.argtypes = [P, ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I), ctypes.POINTER(I)]
        L.tmcs_launch_flow_shape.argtypes = [P] + [ctypes.POINTER(I)] * 4
        L.tmcs_measure_peaks.argtypes = [P]
        L.tmcs_server_open.argtypes = [P, ctypes.POINTER(P)]
        L.tmcs_server_submit.argtypes = [P, P, U64, U64, ctypes.POINTER(ctypes.c_uint64)]
        L.tmcs_server_poll.argtypes = [P, U64, ctypes.POINTER(ctypes.c_int)]
        L.tmcs_server_fetch.argtypes = [P, U64, P, P]
        L.tmcs_server_release.argtypes = [P, U64]
        L.tmcs_server_get_stats.argtypes = [P, P]
        L.tmcs_server_close.argtypes = [P]
        L.tmcs_last_error.argtypes = []
        L.tmcs_last_error.restype = ctypes.c_char_p
        for f in ("tmcs_circuit_build", "tmcs_circuit_free", "tmcs_circuit_info", "tmcs_circuit_stats",
                  "tmcs_reference_sample", "tmcs_sample", "tmcs_sample_range", "tmcs_batch_sample",
                  "tmcs_debug_gap_table", "tmcs_check_device", "tmcs_sample_noalloc", "tmcs_server_open",
                  "tmcs_server_submit", "tmcs_server_poll", "tmcs_server_fetch", "tmcs_server_release",
                  "tmcs_server_get_stats", "tmcs_server_close", "tmcs_fault_count", "tmcs_fault_signatures",
                  "tmcs_sample_measurements", "tmcs_fault_outputs", "tmcs_launch_shape", "tmcs_measure_peaks",
                  "tmcs_dem_columns", "tmcs_launch_flow_shape", "tmcs_debug_gap_counts"):
            getattr(L, f).restype = I
        _lib = L
    return _lib


def tmcs_last_error() -> str:
    return lib().tmcs_last_error().decode()


def _check(rc: int) -> None:
    if rc != TMCS_OK:
        raise TmcsError(rc, tmcs_last_error())


def marshal_ops(circuit: Circuit) -> Tuple[np.ndarray, np.ndarray]:
    """Op list -> (tmcs_op structured array, flat uint32 targets it points into)."""
    ops = circuit.ops
    lens = np.fromiter((o.targets.size for o in ops), dtype=np.int64, count=len(ops))
    flat = (np.concatenate([o.targets for o in ops]).astype(np.uint32)
            if len(ops) and lens.sum() else np.zeros(1, np.uint32))
    flat = np.ascontiguousarray(flat)
    offs = np.zeros(len(ops), dtype=np.int64)
    if len(ops):
        np.cumsum(lens[:-1], out=offs[1:])
    arr = np.zeros(len(ops), dtype=OP_DTYPE)
    arr["code"] = [OPCODE_ID[o.name] for o in ops]
    arr["n_targets"] = lens
    arr["p"] = [o.p for o in ops]
    arr["arg"] = [o.arg for o in ops]
    arr["arg2"] = [getattr(o, "arg2", 0) for o in ops]
    arr["targets"] = flat.ctypes.data + 4 * offs
    return arr, flat


def tmcs_circuit_build(circuit: Circuit, flags: int = 0) -> int:
    """Compile ``circuit``; returns the opaque handle (int)."""
    arr, flat = marshal_ops(circuit)
    out = ctypes.c_void_p()
    _check(lib().tmcs_circuit_build(arr.ctypes.data if arr.size else None, arr.size, flags,
                                    ctypes.byref(out)))
    del flat
    return int(out.value)


def tmcs_circuit_free(handle: int) -> None:
    _check(lib().tmcs_circuit_free(ctypes.c_void_p(handle)))


def tmcs_circuit_info(handle: int) -> Dict[str, int]:
    v = [ctypes.c_uint64() for _ in range(5)]
    _check(lib().tmcs_circuit_info(ctypes.c_void_p(handle), *[ctypes.byref(x) for x in v]))
    return dict(zip(("n_qubits", "n_meas", "n_det", "n_obs", "device_bytes"), (x.value for x in v)))


def tmcs_circuit_stats(handle: int) -> Dict[str, int]:
    s = _Stats()
    _check(lib().tmcs_circuit_stats(ctypes.c_void_p(handle), ctypes.byref(s)))
    return {f: getattr(s, f) for f in STATS_FIELDS}


def tmcs_reference_sample(handle: int) -> np.ndarray:
    """Noiseless reference record as a uint8 array of bits (one per record)."""
    n = tmcs_circuit_info(handle)["n_meas"]
    buf = np.zeros(max((n + 7) // 8, 1), dtype=np.uint8)
    _check(lib().tmcs_reference_sample(ctypes.c_void_p(handle), buf.ctypes.data))
    return np.unpackbits(buf, bitorder="little")[:n]


def tmcs_fault_count(handle: int) -> int:
    n = ctypes.c_uint64()
    _check(lib().tmcs_fault_count(ctypes.c_void_p(handle), ctypes.byref(n)))
    return n.value


def tmcs_fault_outputs(handle: int, fault: int) -> Tuple[List[int], List[int]]:
    """(detectors, observables) flipped by one elementary fault, from the
    host event-signature table."""
    cap = 64
    while True:
        buf = np.zeros(cap, dtype=np.uint32)
        n = ctypes.c_uint32()
        _check(lib().tmcs_fault_outputs(ctypes.c_void_p(handle), fault, buf.ctypes.data, cap, ctypes.byref(n)))
        if n.value <= cap:
            v = [int(x) for x in buf[:n.value]]
            return [x for x in v if x < 0x80000000], [x & 0x7FFFFFFF for x in v if x >= 0x80000000]
        cap = n.value


def tmcs_fault_signatures(handle: int, first_fault: int, n_faults: int, det, obs, stream=None) -> None:
    info = tmcs_circuit_info(handle)
    cols = (n_faults + 63) // 64
    _check_size(det, info["n_det"], cols, "detector")
    _check_size(obs, info["n_obs"], cols, "observable")
    _check(lib().tmcs_fault_signatures(ctypes.c_void_p(handle), first_fault, n_faults, _dev_ptr(det),
                                       _dev_ptr(obs), _stream_ptr(stream)))


def tmcs_dem_columns(handle: int) -> Tuple[List[Tuple[List[int], List[int]]], np.ndarray, np.ndarray]:
    """Detector error model columns (C: tmcs_dem_columns): a list of
    (detectors, observables) per distinct non-empty single-fault signature,
    in the library's canonical order, with each column's probability and
    merged fault count."""
    nc, ne = ctypes.c_uint64(0), ctypes.c_uint64(0)
    h = ctypes.c_void_p(handle)
    _check(lib().tmcs_dem_columns(h, ctypes.byref(nc), ctypes.byref(ne), None, None, None, None))
    off = np.zeros(nc.value + 1, dtype=np.uint64)
    ent = np.zeros(max(ne.value, 1), dtype=np.uint32)
    p = np.zeros(max(nc.value, 1), dtype=np.float64)
    nf = np.zeros(max(nc.value, 1), dtype=np.uint64)
    _check(lib().tmcs_dem_columns(h, ctypes.byref(nc), ctypes.byref(ne), off.ctypes.data, ent.ctypes.data,
                                  p.ctypes.data, nf.ctypes.data))
    cols = []
    for c in range(nc.value):
        v = ent[int(off[c]):int(off[c + 1])]
        cols.append(([int(x) for x in v if x < 0x80000000], [int(x) & 0x7FFFFFFF for x in v if x >= 0x80000000]))
    return cols, p[: nc.value], nf[: nc.value]


def tmcs_check_device() -> None:
    """Raise TmcsError(TMCS_E_TIMEOUT) if a kernel on the current device gave
    up on a bounded wait since the last check."""
    _check(lib().tmcs_check_device())


def tmcs_debug_gap_table(p: float) -> np.ndarray:
    t = np.zeros(4096, dtype=np.uint32)
    _check(lib().tmcs_debug_gap_table(float(p), t.ctypes.data))
    return t


def tmcs_debug_gap_counts(p: float, words, method: int = 0, stream=None):
    """Gap counts of `words` (a CUDA uint32 tensor, or int32 viewed as such)
    for probability p by the device routine `method` (0 the decoupled
    kernel's walkers, 1 the two-read count, 2 kernels 3-6); returns an int32
    CUDA tensor."""
    import torch
    if not (isinstance(words, torch.Tensor) and words.is_cuda and words.is_contiguous() and
            words.element_size() == 4):
        raise ValueError("words must be a contiguous 4-byte CUDA tensor")
    counts = torch.empty(words.shape, dtype=torch.int32, device=words.device)
    _check(lib().tmcs_debug_gap_counts(float(p), words.data_ptr(), words.numel(), counts.data_ptr(), int(method),
                                       _stream_ptr(stream)))
    return counts


def _dev_ptr(buf) -> Optional[int]:
    if buf is None:
        return None
    if isinstance(buf, int):
        return buf
    import torch
    if not isinstance(buf, torch.Tensor):
        raise TypeError("device buffers must be torch CUDA tensors or raw pointers")
    if not buf.is_cuda:
        raise ValueError("device buffer is not a CUDA tensor")
    if not buf.is_contiguous() or buf.element_size() != 8:
        raise ValueError("device buffer must be a contiguous 8-byte-element tensor")
    return buf.data_ptr()


def _stream_ptr(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream or None
    if isinstance(stream, int):
        return stream or None
    return stream.cuda_stream or None


def _check_size(buf, rows: int, cols: int, what: str) -> None:
    if buf is None or isinstance(buf, int):
        return
    if buf.numel() < rows * cols:
        raise ValueError(f"{what} buffer has {buf.numel()} words, needs {rows * cols}")


def tmcs_sample(handle: int, shots: int, seed: int, det, obs, stream=None) -> None:
    info = tmcs_circuit_info(handle)
    cols = (shots + 63) // 64
    _check_size(det, info["n_det"], cols, "detector")
    _check_size(obs, info["n_obs"], cols, "observable")
    _check(lib().tmcs_sample(ctypes.c_void_p(handle), shots, seed & (2 ** 64 - 1), _dev_ptr(det),
                             _dev_ptr(obs), _stream_ptr(stream)))


def tmcs_sample_range(handle: int, first_chunk: int, shots: int, seed: int, det, obs, stream=None) -> None:
    info = tmcs_circuit_info(handle)
    cols = (shots + 63) // 64
    _check_size(det, info["n_det"], cols, "detector")
    _check_size(obs, info["n_obs"], cols, "observable")
    _check(lib().tmcs_sample_range(ctypes.c_void_p(handle), first_chunk, shots, seed & (2 ** 64 - 1),
                                   _dev_ptr(det), _dev_ptr(obs), _stream_ptr(stream)))


def tmcs_sample_noalloc(handle: int, first_chunk: int, shots: int, seed: int, det, obs, stream=None) -> None:
    """Allocation-free sampling (see include/tmcs.h): same bits as
    tmcs_sample_range; its scratch is a fixed 8 MiB device array shared by
    all calls, so calls overlapping on the GPU race."""
    info = tmcs_circuit_info(handle)
    cols = (shots + 63) // 64
    _check_size(det, info["n_det"], cols, "detector")
    _check_size(obs, info["n_obs"], cols, "observable")
    _check(lib().tmcs_sample_noalloc(ctypes.c_void_p(handle), first_chunk, shots, seed & (2 ** 64 - 1),
                                     _dev_ptr(det), _dev_ptr(obs), _stream_ptr(stream)))


def tmcs_sample_measurements(handle: int, first_chunk: int, shots: int, seed: int, meas, stream=None) -> None:
    """Raw measurement records (n_meas rows of ceil(shots/64) words), same
    noise draws as tmcs_sample_range with these arguments plus gauge Paulis
    that make non-deterministic outcomes fair coins (see include/tmcs.h)."""
    info = tmcs_circuit_info(handle)
    cols = (shots + 63) // 64
    _check_size(meas, info["n_meas"], cols, "measurement")
    _check(lib().tmcs_sample_measurements(ctypes.c_void_p(handle), first_chunk, shots, seed & (2 ** 64 - 1),
                                          _dev_ptr(meas), _stream_ptr(stream)))


KERNEL_NAMES = {3: "frame_kernel", 4: "frame_kernel_w", 5: "sig_kernel", 6: "sig_pipe_kernel", 7: "flow_kernel"}


def tmcs_launch_shape(handle: int) -> Dict[str, object]:
    """Autotuned launch shape on the current device: mode (0 = not tuned),
    chunks per CTA (or per warp group), CTA size, detector ring of the chosen
    signature schedule (0 for the frame kernels), and the kernel's name."""
    m, k, t, w = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().tmcs_launch_shape(ctypes.c_void_p(handle), ctypes.byref(m), ctypes.byref(k), ctypes.byref(t),
                                   ctypes.byref(w)))
    ap, win, ga, ae = ctypes.c_int(), ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().tmcs_launch_flow_shape(ctypes.c_void_p(handle), ctypes.byref(ap), ctypes.byref(win),
                                        ctypes.byref(ga), ctypes.byref(ae)))
    name = KERNEL_NAMES.get(m.value)
    label = None
    if name:
        extra = f", ring {w.value}" if w.value else ""
        if m.value == 7:
            extra += f", {ap.value} applier warps, window {win.value}" + (", global arena" if ga.value else "")
        label = f"{name}<{k.value}> ({t.value} threads{extra})"
    return {"mode": m.value, "chunks": k.value, "threads": t.value, "ring_window": w.value, "kernel": label,
            "appliers": ap.value, "window": win.value, "global_arena": ga.value, "arena_entries": ae.value}


class _Peaks(ctypes.Structure):
    _fields_ = [("smem_load_bytes_per_s", ctypes.c_double), ("smem_load_wavefronts_per_s", ctypes.c_double),
                ("smem_atomic_lanes_per_s", ctypes.c_double), ("lop3_lanes_per_s", ctypes.c_double),
                ("lop3_warp_inst_per_s", ctypes.c_double), ("sm_clock_mhz", ctypes.c_double),
                ("sms", ctypes.c_int)]


def tmcs_measure_peaks() -> Dict[str, float]:
    """Measured shared-memory load, shared-atomic and LOP3 rates of the
    current device (microbenchmarks; see include/tmcs.h)."""
    p = _Peaks()
    _check(lib().tmcs_measure_peaks(ctypes.byref(p)))
    return {f: getattr(p, f) for f, _ in _Peaks._fields_}


def tmcs_batch_sample(jobs: Sequence[Tuple[int, int, int, object, object]], stream=None) -> None:
    """jobs: (handle, shots, seed, det, obs) tuples."""
    arr = (_Job * max(len(jobs), 1))()
    for i, (h, shots, seed, det, obs) in enumerate(jobs):
        info = tmcs_circuit_info(h)
        cols = (shots + 63) // 64
        _check_size(det, info["n_det"], cols, "detector")
        _check_size(obs, info["n_obs"], cols, "observable")
        arr[i] = _Job(h, shots, seed & (2 ** 64 - 1), _dev_ptr(det), _dev_ptr(obs))
    _check(lib().tmcs_batch_sample(ctypes.byref(arr), len(jobs), _stream_ptr(stream)))


class Sampler:
    """Owns one compiled circuit; allocates output tensors on demand."""

    def __init__(self, circuit: Circuit, flags: int = 0):
        self.circuit = circuit
        self.handle = tmcs_circuit_build(circuit, flags)
        self.info = tmcs_circuit_info(self.handle)

    def stats(self) -> Dict[str, int]:
        return tmcs_circuit_stats(self.handle)

    def alloc(self, shots: int, device="cuda"):
        import torch
        cols = (shots + 63) // 64
        det = torch.empty((self.info["n_det"], cols), dtype=torch.int64, device=device)
        obs = torch.empty((max(self.info["n_obs"], 1), cols), dtype=torch.int64, device=device)
        return det, obs

    def sample(self, shots: int, seed: int, first_chunk: int = 0, stream=None, out=None):
        det, obs = out if out is not None else self.alloc(shots)
        tmcs_sample_range(self.handle, first_chunk, shots, seed, det, obs if self.info["n_obs"] else None,
                          stream)
        return det, obs[: self.info["n_obs"]]

    def reference_sample(self) -> np.ndarray:
        return tmcs_reference_sample(self.handle)

    def close(self) -> None:
        if self.handle:
            tmcs_circuit_free(self.handle)
            self.handle = 0

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching sampling server (``tmcs_server_*``) on the current
    CUDA device. Circuits passed to ``submit`` are compiled handles (ints) or
    ``Sampler`` objects; they must outlive their requests."""

    def __init__(self, arena_bytes: int = 0, n_streams: int = 0, slice_chunks: int = 0):
        cfg = _ServerConfig(n_streams, slice_chunks, arena_bytes)
        out = ctypes.c_void_p()
        _check(lib().tmcs_server_open(ctypes.byref(cfg), ctypes.byref(out)))
        self.handle = out.value
        self._shape: Dict[int, Tuple[int, int, int]] = {}

    def submit(self, circuit, shots: int, seed: int) -> int:
        h = circuit.handle if isinstance(circuit, Sampler) else int(circuit)
        rid = ctypes.c_uint64()
        _check(lib().tmcs_server_submit(ctypes.c_void_p(self.handle), ctypes.c_void_p(h), shots,
                                        seed & (2 ** 64 - 1), ctypes.byref(rid)))
        info = tmcs_circuit_info(h)
        self._shape[rid.value] = (info["n_det"], info["n_obs"], (shots + 63) // 64)
        return rid.value

    def poll(self, request_id: int) -> str:
        st = ctypes.c_int()
        _check(lib().tmcs_server_poll(ctypes.c_void_p(self.handle), request_id, ctypes.byref(st)))
        return REQ_STATES[st.value]

    def fetch(self, request_id: int) -> Tuple[np.ndarray, np.ndarray]:
        """Wait for the request and return (det, obs) as uint64 arrays in the
        tmcs_sample layout; releases its device space."""
        n_det, n_obs, cols = self._shape.pop(request_id)
        det = np.zeros((n_det, cols), dtype=np.uint64)
        obs = np.zeros((n_obs, cols), dtype=np.uint64)
        _check(lib().tmcs_server_fetch(ctypes.c_void_p(self.handle), request_id,
                                       det.ctypes.data if det.size else None, obs.ctypes.data if obs.size else None))
        return det, obs

    def release(self, request_id: int) -> None:
        self._shape.pop(request_id, None)
        _check(lib().tmcs_server_release(ctypes.c_void_p(self.handle), request_id))

    def stats(self) -> Dict[str, float]:
        st = _ServerStats()
        _check(lib().tmcs_server_get_stats(ctypes.c_void_p(self.handle), ctypes.byref(st)))
        return {name: getattr(st, name) for name, _ in SERVER_STATS_FIELDS}

    def close(self) -> None:
        if self.handle:
            _check(lib().tmcs_server_close(ctypes.c_void_p(self.handle)))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
