"""Thin ctypes binding of libpcpd.so (declared in include/pcpd.h).

Argument marshalling only: every step of the sweep runs in the library's CUDA kernels.
There is no CPU fallback; if the library is missing or no CUDA device is usable, the calls
raise.  PyTorch is optional here and only supplies device memory and streams.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# PCPD_LIB may name another build of the library (e.g. libpcpd_debug.so, the index-checked one)
LIB_PATH = os.environ.get("PCPD_LIB") or os.path.join(_HERE, "libpcpd.so")

PCPD_OK, PCPD_EINVAL, PCPD_ENOMEM, PCPD_ECUDA, PCPD_ETIMEOUT, PCPD_ESTATE, PCPD_ENODEV = range(7)
INIT_FULL, INIT_EMPTY, INIT_HALF = 0, 1, 2

_u32p = C.POINTER(C.c_uint32)
_u64p = C.POINTER(C.c_uint64)
_f64p = C.POINTER(C.c_double)


class PcpdError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"pcpd error {code}: {msg}")
        self.code = code


class Params(C.Structure):
    _fields_ = [("L", C.c_uint32), ("samples", C.c_uint32), ("p", C.c_double), ("d", C.c_double),
                ("seed", C.c_uint64), ("init", C.c_int), ("stream", C.c_void_p),
                ("dev_lattice", C.c_void_p), ("dev_bytes", C.c_size_t), ("per_sample", C.c_int),
                ("plan_threads", C.c_uint32), ("plan_seg_sites", C.c_uint32), ("plan_tau", C.c_uint32),
                ("autotune", C.c_int), ("jit", C.c_int), ("tuple", C.c_uint32), ("group0", C.c_uint32)]


class PlanInfo(C.Structure):
    _fields_ = [("ring", C.c_uint32), ("gpi", C.c_uint32), ("threads", C.c_uint32), ("core", C.c_uint32),
                ("halo", C.c_uint32), ("tau", C.c_uint32), ("n_seg", C.c_uint32), ("tiles", C.c_uint32),
                ("grid", C.c_uint32), ("jit", C.c_uint32), ("smem_bytes", C.c_size_t)]


class ServerConfig(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_size_t), ("max_active", C.c_uint32), ("chunk_attempts", C.c_uint64),
                ("stream", C.c_void_p)]


class ServerStats(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("completed", C.c_uint64), ("failed", C.c_uint64),
                ("rounds", C.c_uint64), ("busy_seconds", C.c_double), ("attempts", C.c_ulonglong),
                ("active", C.c_uint64), ("queued", C.c_uint64), ("mem_used_bytes", C.c_size_t)]


class PaperParams(C.Structure):
    _fields_ = [("n_loc", C.c_uint32), ("S_w", C.c_uint32), ("systems", C.c_uint32), ("p", C.c_double),
                ("d", C.c_double), ("m", C.c_uint32), ("n_dec", C.c_uint32), ("seed", C.c_uint64),
                ("init", C.c_int), ("stream", C.c_void_p), ("plan_spc", C.c_uint32), ("generic", C.c_int)]


# (name, restype, argtypes) of every exported entry point in include/pcpd.h
SIGNATURES = [
    ("pcpd_create", C.c_void_p, [C.c_uint32, C.c_uint32, C.c_double, C.c_double, C.c_uint64]),
    ("pcpd_create_ex", C.c_int, [C.POINTER(Params), C.POINTER(C.c_void_p)]),
    ("pcpd_run", C.c_int, [C.c_void_p, C.c_uint64, _u64p, C.c_size_t]),
    ("pcpd_num_records", C.c_size_t, [C.c_void_p]),
    ("pcpd_get_plan", C.c_int, [C.c_void_p, C.POINTER(PlanInfo)]),
    ("pcpd_density", C.c_int, [C.c_void_p, _f64p, _u64p, C.c_size_t]),
    ("pcpd_record_times", C.c_int, [C.c_void_p, _u64p, C.c_size_t]),
    ("pcpd_sample_counts", C.c_int, [C.c_void_p, C.c_size_t, _u32p]),
    ("pcpd_pair_counts", C.c_int, [C.c_void_p, _u64p, C.c_size_t]),
    ("pcpd_pair_density", C.c_int, [C.c_void_p, _f64p, C.c_size_t]),
    ("pcpd_get_lattice", C.c_int, [C.c_void_p, _u32p]),
    ("pcpd_set_lattice", C.c_int, [C.c_void_p, _u32p, C.c_uint64]),
    ("pcpd_get_lattice_async", C.c_int, [C.c_void_p, _u32p]),
    ("pcpd_set_lattice_async", C.c_int, [C.c_void_p, _u32p, C.c_uint64]),
    ("pcpd_run_substeps", C.c_int, [C.c_void_p, C.c_uint64]),
    ("pcpd_substep", C.c_uint64, [C.c_void_p]),
    ("pcpd_time_mcs", C.c_uint64, [C.c_void_p]),
    ("pcpd_sync", C.c_int, [C.c_void_p]),
    ("pcpd_destroy", None, [C.c_void_p]),
    ("pcpd_last_error", C.c_char_p, []),
    ("pcpd_debug_build", C.c_int, []),
    ("pcpd_debug_check", C.c_uint, []),
    ("pcpd_kernel_launches", C.c_ulonglong, []),
    ("pcpd_thresholds", C.c_int, [C.c_double, C.c_double, _u64p, _u64p]),
    ("pcpd_substep_of_time", C.c_uint64, [C.c_uint32, C.c_uint64]),
    ("pcpd_substep_of_time_n", C.c_uint64, [C.c_uint32, C.c_uint32, C.c_uint64]),
    ("pcpd_dev_philox", C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.c_size_t, C.c_void_p]),
    ("pcpd_dev_rate_masks", C.c_int, [C.c_void_p, C.c_uint64, C.c_uint64, C.c_void_p, C.c_size_t, C.c_void_p]),
    ("pcpd_dev_timeout_test", C.c_int, [C.c_ulonglong]),
    ("pcpd_autotune", C.c_int, [C.POINTER(Params), C.c_uint32, C.POINTER(Params), _f64p]),
    ("pcpd_batch_create", C.c_int, [C.c_void_p, C.POINTER(C.c_void_p)]),
    ("pcpd_batch_add", C.c_int, [C.c_void_p, C.POINTER(Params), C.c_uint64, _u64p, C.c_size_t, C.POINTER(C.c_size_t)]),
    ("pcpd_batch_run", C.c_int, [C.c_void_p]),
    ("pcpd_batch_size", C.c_size_t, [C.c_void_p]),
    ("pcpd_batch_set_jit", C.c_int, [C.c_void_p, C.c_int]),
    ("pcpd_batch_jit_launches", C.c_size_t, [C.c_void_p]),
    ("pcpd_batch_counts", C.c_int, [C.c_void_p, C.c_size_t, _u64p, C.c_size_t]),
    ("pcpd_batch_lattice", C.c_int, [C.c_void_p, C.c_size_t, _u32p]),
    ("pcpd_batch_pair_counts", C.c_int, [C.c_void_p, C.c_size_t, _u64p, C.c_size_t]),
    ("pcpd_batch_destroy", None, [C.c_void_p]),
    ("pcpd_server_start", C.c_int, [C.POINTER(ServerConfig), C.POINTER(C.c_void_p)]),
    ("pcpd_server_submit", C.c_int, [C.c_void_p, C.POINTER(Params), C.c_uint64, _u64p, C.c_size_t, C.c_int,
                                     C.POINTER(C.c_uint64)]),
    ("pcpd_server_poll", C.c_int, [C.c_void_p, C.c_uint64, C.POINTER(C.c_int)]),
    ("pcpd_server_cancel", C.c_int, [C.c_void_p, C.c_uint64]),
    ("pcpd_server_result", C.c_int, [C.c_void_p, C.c_uint64, _u64p, C.c_size_t, _u32p, _f64p, _f64p]),
    ("pcpd_server_wait_idle", C.c_int, [C.c_void_p]),
    ("pcpd_server_get_stats", C.c_int, [C.c_void_p, C.POINTER(ServerStats)]),
    ("pcpd_server_stop", None, [C.c_void_p]),
    ("pcpd_paper_thresholds", C.c_int, [C.c_double, C.c_double, C.c_uint32, C.c_uint32, _u32p, _u64p]),
    ("pcpd_paper_create", C.c_int, [C.POINTER(PaperParams), C.POINTER(C.c_void_p)]),
    ("pcpd_paper_run", C.c_int, [C.c_void_p, C.c_uint64, _u64p, C.c_size_t]),
    ("pcpd_paper_num_records", C.c_size_t, [C.c_void_p]),
    ("pcpd_paper_step", C.c_uint64, [C.c_void_p]),
    ("pcpd_paper_counts", C.c_int, [C.c_void_p, _u64p, _u32p, C.c_size_t]),
    ("pcpd_paper_get_lattice", C.c_int, [C.c_void_p, _u32p]),
    ("pcpd_paper_set_lattice", C.c_int, [C.c_void_p, _u32p, C.c_uint64]),
    ("pcpd_paper_get_plan", C.c_int, [C.c_void_p, _u32p, _u32p, _u32p, C.POINTER(C.c_size_t)]),
    ("pcpd_paper_sync", C.c_int, [C.c_void_p]),
    ("pcpd_paper_destroy", None, [C.c_void_p]),
    ("pcpd_sweep_noalloc", C.c_int, [C.c_void_p, C.c_void_p, C.c_uint32, C.c_uint32, C.c_double, C.c_double,
                                     C.c_uint64, C.c_uint64, C.c_uint64, C.c_void_p]),
]

_lib = None


def load(path: str = LIB_PATH):
    """Load libpcpd.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError(f"{path} is missing: build it with paper_1301_6082_gb300.build.build()")
        lib = C.CDLL(path)
        for name, res, args in SIGNATURES:
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _check(rc: int):
    if rc != PCPD_OK:
        raise PcpdError(rc, load().pcpd_last_error().decode())


def kernel_launches() -> int:
    return int(load().pcpd_kernel_launches())


def thresholds(p: float, d: float):
    td, tda = C.c_uint64(), C.c_uint64()
    _check(load().pcpd_thresholds(p, d, C.byref(td), C.byref(tda)))
    return int(td.value), int(tda.value)


def substep_of_time(L: int, t: int, tuple_n: int = 2) -> int:
    if tuple_n == 2:
        return int(load().pcpd_substep_of_time(L, t))
    return int(load().pcpd_substep_of_time_n(L, tuple_n, t))


def _ptr(a: np.ndarray, t):
    return a.ctypes.data_as(C.POINTER(t))


class Pcpd:
    """One simulation handle: `samples` bit-sliced PCPD samples on a ring of L sites
    (tuple_n = 3 / 4: the TCPD / QCPD, reacting triplets / quadruplets)."""

    def __init__(self, L: int, samples: int, p: float, d: float, seed: int = 1,
                 init: int = INIT_FULL, per_sample: bool = False, stream=None,
                 dev_lattice=None, plan_threads: int = 0, plan_seg_sites: int = 0,
                 plan_tau: int = 0, autotune: bool = False, jit: int = 0, tuple_n: int = 2,
                 group0: int = 0):
        lib = load()
        prm = Params()
        prm.L, prm.samples, prm.p, prm.d, prm.seed, prm.init = L, samples, p, d, seed, init
        prm.per_sample = 1 if per_sample else 0
        prm.plan_threads, prm.plan_seg_sites, prm.plan_tau = plan_threads, plan_seg_sites, plan_tau
        prm.autotune = 1 if autotune else 0
        prm.jit = jit
        prm.tuple = tuple_n
        prm.group0 = group0
        if stream is not None:
            prm.stream = C.c_void_p(int(getattr(stream, "cuda_stream", stream)))
        self._keep = dev_lattice
        if dev_lattice is not None:   # a torch CUDA tensor (or any object with data_ptr/nbytes)
            prm.dev_lattice = C.c_void_p(int(dev_lattice.data_ptr()))
            prm.dev_bytes = int(dev_lattice.numel() * dev_lattice.element_size())
        h = C.c_void_p()
        _check(lib.pcpd_create_ex(C.byref(prm), C.byref(h)))
        self._h = h
        self.L, self.S, self.p, self.d, self.seed = L, samples, p, d, seed
        self.G = samples // 32
        self.tuple_n = tuple_n

    def close(self):
        if getattr(self, "_h", None):
            load().pcpd_destroy(self._h)
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

    def run(self, steps_mcs: int, record_times=()):
        t = np.ascontiguousarray(record_times, dtype=np.uint64)
        _check(load().pcpd_run(self._h, steps_mcs, _ptr(t, C.c_uint64) if t.size else None, t.size))

    def run_substeps(self, n: int):
        _check(load().pcpd_run_substeps(self._h, n))

    @property
    def num_records(self) -> int:
        return int(load().pcpd_num_records(self._h))

    @property
    def substep(self) -> int:
        return int(load().pcpd_substep(self._h))

    @property
    def time_mcs(self) -> int:
        return int(load().pcpd_time_mcs(self._h))

    def counts(self) -> np.ndarray:
        n = self.num_records
        c = np.zeros(n, dtype=np.uint64)
        if n:
            _check(load().pcpd_density(self._h, None, _ptr(c, C.c_uint64), n))
        return c

    def pair_counts(self) -> np.ndarray:
        """Occupied nearest-neighbour pairs per record, summed over samples."""
        n = self.num_records
        c = np.zeros(n, dtype=np.uint64)
        if n:
            _check(load().pcpd_pair_counts(self._h, _ptr(c, C.c_uint64), n))
        return c

    def pair_density(self) -> np.ndarray:
        """Occupied nearest-neighbour pairs per site and sample, per record (Sec. 5.3)."""
        n = self.num_records
        r = np.zeros(n, dtype=np.float64)
        if n:
            _check(load().pcpd_pair_density(self._h, _ptr(r, C.c_double), n))
        return r

    def density(self) -> np.ndarray:
        n = self.num_records
        r = np.zeros(n, dtype=np.float64)
        if n:
            _check(load().pcpd_density(self._h, _ptr(r, C.c_double), None, n))
        return r

    def record_times(self) -> np.ndarray:
        n = self.num_records
        t = np.zeros(n, dtype=np.uint64)
        if n:
            _check(load().pcpd_record_times(self._h, _ptr(t, C.c_uint64), n))
        return t

    def sample_counts(self, r: int) -> np.ndarray:
        out = np.zeros(self.S, dtype=np.uint32)
        _check(load().pcpd_sample_counts(self._h, r, _ptr(out, C.c_uint32)))
        return out

    def lattice(self, out: np.ndarray | None = None, wait: bool = True) -> np.ndarray:
        """Copy the lattice ([G][L] uint32) into `out` (a new array if None).  wait=False
        enqueues the copy on the handle's stream (keep `out` alive, ideally page-locked, and
        call sync() before reading it)."""
        if out is None:
            out = np.zeros((self.G, self.L), dtype=np.uint32)
        assert out.dtype == np.uint32 and out.shape == (self.G, self.L) and out.flags.c_contiguous
        fn = load().pcpd_get_lattice if wait else load().pcpd_get_lattice_async
        _check(fn(self._h, _ptr(out, C.c_uint32)))
        return out

    def set_lattice(self, words: np.ndarray, substep: int, wait: bool = True):
        """Replace the lattice; wait=False enqueues the copy (`words` must be a C-contiguous
        uint32 [G][L] array that stays unchanged until the stream has passed the copy)."""
        if wait:
            w = np.ascontiguousarray(words, dtype=np.uint32)
        else:
            w = words
            assert w.dtype == np.uint32 and w.flags.c_contiguous
        assert w.shape == (self.G, self.L)
        fn = load().pcpd_set_lattice if wait else load().pcpd_set_lattice_async
        _check(fn(self._h, _ptr(w, C.c_uint32), substep))

    def sync(self):
        _check(load().pcpd_sync(self._h))

    def plan(self) -> dict:
        info = PlanInfo()
        _check(load().pcpd_get_plan(self._h, C.byref(info)))
        return {f: getattr(info, f) for f, _ in PlanInfo._fields_}


class Batch:
    """Many independent instances run by one persistent launch (pcpd_batch_*)."""

    def __init__(self, stream=None):
        h = C.c_void_p()
        s = C.c_void_p(int(getattr(stream, "cuda_stream", stream))) if stream is not None else None
        _check(load().pcpd_batch_create(s, C.byref(h)))
        self._h = h
        self._meta = []

    def add(self, L: int, samples: int, p: float, d: float, seed: int, steps_mcs: int,
            record_times=(), init: int = INIT_FULL, plan_threads: int = 0, plan_seg_sites: int = 0,
            plan_tau: int = 0, tuple_n: int = 2, group0: int = 0) -> int:
        prm = Params()
        prm.L, prm.samples, prm.p, prm.d, prm.seed, prm.init = L, samples, p, d, seed, init
        prm.plan_threads, prm.plan_seg_sites, prm.plan_tau = plan_threads, plan_seg_sites, plan_tau
        prm.tuple = tuple_n
        prm.group0 = group0
        t = np.ascontiguousarray(record_times, dtype=np.uint64)
        idx = C.c_size_t()
        _check(load().pcpd_batch_add(self._h, C.byref(prm), steps_mcs, _ptr(t, C.c_uint64) if t.size else None,
                                     t.size, C.byref(idx)))
        self._meta.append((L, samples, len(t)))
        return int(idx.value)

    def set_jit(self, mode: int):
        """Runtime-specialised kernels for members sharing a threshold pair: 1 always, 0 when
        their work is large enough, -1 never (include/pcpd.h, pcpd_batch_set_jit)."""
        _check(load().pcpd_batch_set_jit(self._h, mode))

    @property
    def jit_launches(self) -> int:
        return int(load().pcpd_batch_jit_launches(self._h))

    def run(self):
        _check(load().pcpd_batch_run(self._h))

    def counts(self, i: int) -> np.ndarray:
        n = self._meta[i][2]
        c = np.zeros(n, dtype=np.uint64)
        if n:
            _check(load().pcpd_batch_counts(self._h, i, _ptr(c, C.c_uint64), n))
        return c

    def pair_counts(self, i: int) -> np.ndarray:
        n = self._meta[i][2]
        c = np.zeros(n, dtype=np.uint64)
        if n:
            _check(load().pcpd_batch_pair_counts(self._h, i, _ptr(c, C.c_uint64), n))
        return c

    def lattice(self, i: int) -> np.ndarray:
        L, S, _ = self._meta[i]
        out = np.zeros((S // 32, L), dtype=np.uint32)
        _check(load().pcpd_batch_lattice(self._h, i, _ptr(out, C.c_uint32)))
        return out

    def close(self):
        if getattr(self, "_h", None):
            load().pcpd_batch_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request loop of the library (pcpd_server_*)."""

    def __init__(self, hbm_budget_bytes: int = 64 << 30, max_active: int = 128,
                 chunk_attempts: int = 1 << 31, stream=None):
        cfg = ServerConfig()
        cfg.hbm_budget_bytes, cfg.max_active, cfg.chunk_attempts = hbm_budget_bytes, max_active, chunk_attempts
        if stream is not None:
            cfg.stream = C.c_void_p(int(getattr(stream, "cuda_stream", stream)))
        h = C.c_void_p()
        _check(load().pcpd_server_start(C.byref(cfg), C.byref(h)))
        self._h = h
        self._meta = {}

    def submit(self, L: int, samples: int, p: float, d: float, seed: int, steps_mcs: int,
               record_times=(), init: int = INIT_FULL, keep_lattice: bool = False, tuple_n: int = 2,
               group0: int = 0) -> int:
        prm = Params()
        prm.L, prm.samples, prm.p, prm.d, prm.seed, prm.init = L, samples, p, d, seed, init
        prm.tuple = tuple_n
        prm.group0 = group0
        t = np.ascontiguousarray(record_times, dtype=np.uint64)
        rid = C.c_uint64()
        _check(load().pcpd_server_submit(self._h, C.byref(prm), steps_mcs, _ptr(t, C.c_uint64) if t.size else None,
                                         t.size, 1 if keep_lattice else 0, C.byref(rid)))
        self._meta[int(rid.value)] = (L, samples, len(t), keep_lattice)
        return int(rid.value)

    def cancel(self, rid: int):
        """Cancel a queued or running request (it then fails with "cancelled")."""
        _check(load().pcpd_server_cancel(self._h, rid))

    def poll(self, rid: int) -> int:
        st = C.c_int()
        _check(load().pcpd_server_poll(self._h, rid, C.byref(st)))
        return int(st.value)

    def result(self, rid: int):
        """(counts, lattice or None, latency_s, queue_s) of a request (waits for it)."""
        L, S, n, keep = self._meta[rid]
        c = np.zeros(n, dtype=np.uint64)
        lat = np.zeros((S // 32, L), dtype=np.uint32) if keep else None
        latency, queue = C.c_double(), C.c_double()
        _check(load().pcpd_server_result(self._h, rid, _ptr(c, C.c_uint64) if n else None, n,
                                         _ptr(lat, C.c_uint32) if keep else None, C.byref(latency), C.byref(queue)))
        return c, lat, latency.value, queue.value

    def wait_idle(self):
        _check(load().pcpd_server_wait_idle(self._h))

    def stats(self) -> dict:
        st = ServerStats()
        _check(load().pcpd_server_get_stats(self._h, C.byref(st)))
        return {f: getattr(st, f) for f, _ in ServerStats._fields_}

    def stop(self):
        if getattr(self, "_h", None):
            load().pcpd_server_stop(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.stop()

    def __del__(self):
        try:
            self.stop()
        except Exception:
            pass


def autotune(L: int, samples: int, p: float, d: float, seed: int = 1, trial_substeps: int = 0,
             tuple_n: int = 2):
    """Fastest plan for (L, samples): dict(plan_threads, plan_seg_sites, plan_tau, rate)."""
    prm = Params()
    prm.L, prm.samples, prm.p, prm.d, prm.seed = L, samples, p, d, seed
    prm.tuple = tuple_n
    best = Params()
    rate = C.c_double()
    _check(load().pcpd_autotune(C.byref(prm), trial_substeps, C.byref(best), C.byref(rate)))
    return {"plan_threads": best.plan_threads, "plan_seg_sites": best.plan_seg_sites,
            "plan_tau": best.plan_tau, "rate": rate.value}


def dev_timeout_test(spin_limit_cycles: int) -> int:
    """Return code of the engine's failure-path test (PCPD_ETIMEOUT when it behaves)."""
    return int(load().pcpd_dev_timeout_test(spin_limit_cycles))


def dev_philox(ctr_dev, seed: int, out_dev, n: int, stream=None):
    """Device Philox on torch CUDA tensors ctr_dev / out_dev (uint32-compatible, [n,4])."""
    s = C.c_void_p(int(getattr(stream, "cuda_stream", 0) or 0)) if stream is not None else None
    _check(load().pcpd_dev_philox(C.c_void_p(ctr_dev.data_ptr()), seed, C.c_void_p(out_dev.data_ptr()), n, s))


def dev_rate_masks(words_dev, t_d: int, t_da: int, masks_dev, n: int, stream=None):
    s = C.c_void_p(int(getattr(stream, "cuda_stream", 0) or 0)) if stream is not None else None
    _check(load().pcpd_dev_rate_masks(C.c_void_p(words_dev.data_ptr()), t_d, t_da,
                                      C.c_void_p(masks_dev.data_ptr()), n, s))


def check_noalloc_buffers(lat_in_dev, lat_out_dev, L: int, samples: int):
    """The C entry point cannot see how large the caller's buffers are: refuse, before any
    launch, buffers that are not contiguous CUDA tensors on the current device holding at
    least (samples/32)*L uint32 words each."""
    need = (samples // 32) * L * 4
    bufs = (("lat_in", lat_in_dev), ("lat_out", lat_out_dev))
    for name, t in bufs:
        if not getattr(t, "is_cuda", False):
            raise PcpdError(PCPD_EINVAL, f"{name} must be a CUDA tensor")
        if not t.is_contiguous():
            raise PcpdError(PCPD_EINVAL, f"{name} must be contiguous")
        have = t.numel() * t.element_size()
        if have < need:
            raise PcpdError(PCPD_EINVAL, f"{name} holds {have} bytes, the lattice needs {need}")
    import torch
    cur = torch.cuda.current_device()
    for name, t in bufs:
        if t.device.index != cur:
            raise PcpdError(PCPD_EINVAL, f"{name} is on cuda:{t.device.index}, the current device is cuda:{cur}")


def sweep_noalloc(lat_in_dev, lat_out_dev, L: int, samples: int, p: float, d: float, seed: int,
                  substep_begin: int, n_substeps: int, stream=None):
    """Allocation-free sweep on caller-owned device lattices (torch CUDA tensors or objects
    with data_ptr()): lat_out receives the state after n_substeps more sub-steps; lat_in is
    used as work space.  For callers that cannot let the library allocate device memory."""
    check_noalloc_buffers(lat_in_dev, lat_out_dev, L, samples)
    s = C.c_void_p(int(getattr(stream, "cuda_stream", 0) or 0)) if stream is not None else None
    _check(load().pcpd_sweep_noalloc(C.c_void_p(lat_in_dev.data_ptr()), C.c_void_p(lat_out_dev.data_ptr()),
                                     L, samples, p, d, seed, substep_begin, n_substeps, s))


def paper_thresholds(p: float, d: float, m: int, n_dec: int):
    """(T_d, T_c) of the paper's scheme (see include/pcpd.h)."""
    td, tc = C.c_uint32(), C.c_uint64()
    _check(load().pcpd_paper_thresholds(p, d, m, n_dec, C.byref(td), C.byref(tc)))
    return int(td.value), int(tc.value)


class PaperScheme:
    """The paper's own GPU scheme (Sec. 3-4, Alg. 2): `systems` independent rings of
    L = 32*n_loc*S_w sites, one group of S_w threads each, a shared random local site per
    step, dyadic diffusion masks and correlated annihilation draws with n_dec decorrelation
    words.  Lattice layout: words [systems][n_loc][S_w]; bit b of [s][l][w] is site
    b*(L/32) + w*n_loc + l.  Time in steps: one MCS = n_loc steps."""

    def __init__(self, n_loc: int, S_w: int, systems: int, p: float, d: float, m: int = 1,
                 n_dec: int = 2, seed: int = 1, init: int = INIT_FULL, stream=None,
                 plan_spc: int = 0, generic: bool = False):
        lib = load()
        prm = PaperParams()
        prm.n_loc, prm.S_w, prm.systems, prm.p, prm.d = n_loc, S_w, systems, p, d
        prm.m, prm.n_dec, prm.seed, prm.init = m, n_dec, seed, init
        prm.plan_spc, prm.generic = plan_spc, 1 if generic else 0
        if stream is not None:
            prm.stream = C.c_void_p(int(getattr(stream, "cuda_stream", stream)))
        h = C.c_void_p()
        _check(lib.pcpd_paper_create(C.byref(prm), C.byref(h)))
        self._h = h
        self.n_loc, self.S_w, self.systems = n_loc, S_w, systems
        self.L = 32 * n_loc * S_w

    def close(self):
        if getattr(self, "_h", None):
            load().pcpd_paper_destroy(self._h)
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

    def run(self, n_steps: int, record_steps=()):
        r = np.ascontiguousarray(record_steps, dtype=np.uint64)
        _check(load().pcpd_paper_run(self._h, n_steps, _ptr(r, C.c_uint64) if r.size else None, r.size))

    @property
    def step(self) -> int:
        return int(load().pcpd_paper_step(self._h))

    @property
    def num_records(self) -> int:
        return int(load().pcpd_paper_num_records(self._h))

    def counts(self, per_system: bool = False):
        n = self.num_records
        c = np.zeros(n, dtype=np.uint64)
        ps = np.zeros((n, self.systems), dtype=np.uint32) if per_system else None
        if n:
            _check(load().pcpd_paper_counts(self._h, _ptr(c, C.c_uint64),
                                            _ptr(ps, C.c_uint32) if ps is not None else None, n))
        return (c, ps) if per_system else c

    def density(self) -> np.ndarray:
        return self.counts() / float(self.L * self.systems)

    def lattice(self) -> np.ndarray:
        out = np.zeros((self.systems, self.n_loc, self.S_w), dtype=np.uint32)
        _check(load().pcpd_paper_get_lattice(self._h, _ptr(out, C.c_uint32)))
        return out

    def set_lattice(self, words: np.ndarray, step: int):
        w = np.ascontiguousarray(words, dtype=np.uint32)
        assert w.shape == (self.systems, self.n_loc, self.S_w)
        _check(load().pcpd_paper_set_lattice(self._h, _ptr(w, C.c_uint32), step))

    def plan(self) -> dict:
        a, b, c, s = C.c_uint32(), C.c_uint32(), C.c_uint32(), C.c_size_t()
        _check(load().pcpd_paper_get_plan(self._h, C.byref(a), C.byref(b), C.byref(c), C.byref(s)))
        return {"systems_per_cta": a.value, "threads": b.value, "grid": c.value, "smem_bytes": s.value}

    def sync(self):
        _check(load().pcpd_paper_sync(self._h))


def debug_build() -> bool:
    """True when the loaded library is the index-checked debug build."""
    return bool(load().pcpd_debug_build())


def debug_check() -> int:
    """First failed index check since the last call (0: none), in debug builds; 0 otherwise."""
    return int(load().pcpd_debug_check())
