"""Thin Python binding of the DZS TreePM C ABI (include/dzs.h).

Argument marshalling only: every step of the method runs in the CUDA kernels of
libdzs.so (built for sm_103a by ``paper_2005_05328_gb300.build``).  There is no
CPU fallback: if the library is missing or the device is not a GB300 the calls
raise.  Function names match the C entry points (``dzs_create`` ...); the
``Context`` class bundles them for convenience.

Paper: Garaldi, Nori & Baldi, "Dynamic Zoom Simulations", arXiv 2005.05328.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libdzs.so")

DZS_OK, DZS_EINVAL, DZS_ENOMEM, DZS_ECUDA, DZS_EOVERFLOW, DZS_ETIMEOUT, DZS_ESTATE, DZS_EDEVICE = range(8)
STATUS_NAMES = ["DZS_OK", "DZS_EINVAL", "DZS_ENOMEM", "DZS_ECUDA", "DZS_EOVERFLOW", "DZS_ETIMEOUT",
                "DZS_ESTATE", "DZS_EDEVICE"]
RLC_SWEEP, RLC_PHYSICAL = 0, 1
FP32, FP64 = 0, 1
CRIT_GEOMETRIC, CRIT_DYNAMICAL = 0, 1
WALK_AUTO, WALK_MASKED, WALK_GUARDED = 0, 1, 2
FL_CROSSED, FL_MERGED = 1, 2
STAGE_KICK_DRIFT, STAGE_SORT, STAGE_MERGE, STAGE_FORCE, STAGE_CLOSE, STAGE_ALL = 1, 2, 4, 8, 16, 31
ACC_PM, ACC_TREE, ACC_ALL = 1, 2, 3
MESH_DELTA, MESH_PHI = 0, 1
PK_SHOT = 1

EXPORTED = ["dzs_params_default", "dzs_footprint_bytes", "dzs_create", "dzs_ics", "dzs_step",
            "dzs_run_stages", "dzs_lightcone_drain", "dzs_pipeline", "dzs_step_result", "dzs_lightcone_drain_step",
            "dzs_destroy", "dzs_get_count", "dzs_get_state",
            "dzs_set_state", "dzs_accel", "dzs_merge_only", "dzs_diagnostics", "dzs_get_tables",
            "dzs_get_mesh", "dzs_get_counters", "dzs_get_walk_counters", "dzs_walk_lists", "dzs_measure_fp32_peaks", "dzs_debug_fail_alloc", "dzs_twin_displacement", "dzs_batch_create", "dzs_batch_step",
            "dzs_batch_synchronize", "dzs_batch_destroy", "dzs_set_profiling", "dzs_get_profile",
            "dzs_morton_sort_noalloc", "dzs_checkpoint_bytes", "dzs_checkpoint", "dzs_restore",
            "dzs_step_until", "dzs_observe_enable", "dzs_observe_add_records", "dzs_skymap_get",
            "dzs_lcdensity_get", "dzs_skymap_alm", "dzs_power_spectrum", "dzs_serve", "dzs_fof", "dzs_last_error"]
NOALLOC_SORT_MAX_N = 262144
PROF_NAMES = ["kick_drift", "sort", "merge", "tree", "pm", "walk", "fft"]


class Params(C.Structure):
    _fields_ = [
        ("n1d", C.c_int32), ("mesh", C.c_int32), ("box", C.c_double),
        ("omega_m", C.c_double), ("omega_l", C.c_double), ("hubble", C.c_double),
        ("sigma8", C.c_double), ("ns", C.c_double), ("z_init", C.c_double),
        ("nsteps", C.c_int32), ("leaf_bucket", C.c_int32), ("walk_group", C.c_int32),
        ("dzs_on", C.c_int32), ("merge_level", C.c_int32), ("rlc_mode", C.c_int32),
        ("rs_cells", C.c_double), ("rcut_rs", C.c_double), ("theta", C.c_double),
        ("soft_frac", C.c_double), ("theta_dzs", C.c_double), ("buffer_cells", C.c_double),
        ("seed", C.c_uint64), ("precision", C.c_int32), ("device", C.c_int32),
        ("lc_capacity", C.c_uint64), ("dzs_criterion", C.c_int32), ("walk_eval", C.c_int32),
        ("alpha_dyn", C.c_double), ("capacity", C.c_uint64),
    ]


class Halt(C.Structure):
    _fields_ = [("ratio_min", C.c_double), ("wall_limit_s", C.c_double), ("horizon_s", C.c_double)]


HALT_NONE, HALT_RATIO, HALT_PREDICTED, HALT_WALL = 0, 1, 2, 3


class Request(C.Structure):
    _fields_ = [("arrival_s", C.c_double), ("n1d", C.c_int32), ("mesh", C.c_int32), ("box", C.c_double),
                ("sigma8", C.c_double), ("seed", C.c_uint64)]


class RequestResult(C.Structure):
    _fields_ = [("admit_s", C.c_double), ("done_s", C.c_double), ("n_end", C.c_uint64),
                ("records", C.c_uint64), ("record_hash", C.c_uint64), ("diag", C.c_double * 8),
                ("status", C.c_int32), ("reserved_", C.c_int32)]


class ServeConfig(C.Structure):
    _fields_ = [("hbm_budget_bytes", C.c_double), ("max_active", C.c_int32), ("steps_per_slice", C.c_int32),
                ("host_threads", C.c_int32), ("reserved_", C.c_int32), ("base", Params)]


class Observe(C.Structure):
    _fields_ = [("nside", C.c_int32), ("mesh", C.c_int32), ("a_lo", C.c_double), ("a_hi", C.c_double)]


HALO_DTYPE = np.dtype([("first", "<i8"), ("count", "<i8"), ("mass", "<u8"), ("x", "<f8", (3,)),
                       ("rmax2", "<u8")])

RECORD_DTYPE = np.dtype([("id", "<u4"), ("k", "<u4"), ("a_cross", "<f8"),
                         ("x", "<f8", (3,)), ("p", "<f8", (3,))])

_lib = None


class DzsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < 8 else status, msg))
        self.status = status


def load(path: str = LIB_PATH):
    """Load libdzs.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError("libdzs.so not built: run paper_2005_05328_gb300.build.build() "
                           "(or __graft_entry__.build()) first")
    L = C.CDLL(path)
    vp, sz, i32, u32, u64 = C.c_void_p, C.c_size_t, C.c_int32, C.c_uint32, C.c_uint64
    P = C.POINTER(Params)
    sig = {
        "dzs_params_default": [P], "dzs_footprint_bytes": [P, C.POINTER(sz)],
        "dzs_create": [P, vp, C.POINTER(vp)], "dzs_ics": [vp],
        "dzs_step": [vp, i32, C.POINTER(i32)], "dzs_run_stages": [vp, u32],
        "dzs_lightcone_drain": [vp, vp, sz, C.POINTER(sz)], "dzs_destroy": [vp],
        "dzs_pipeline": [vp, i32], "dzs_step_result": [vp, i32, vp, C.POINTER(C.c_uint64)],
        "dzs_lightcone_drain_step": [vp, i32, vp, sz, C.POINTER(sz)],
        "dzs_get_count": [vp, C.POINTER(sz), C.POINTER(i32)],
        "dzs_get_state": [vp, vp, vp, vp, vp, vp, vp, sz, C.POINTER(sz)],
        "dzs_set_state": [vp, vp, vp, vp, vp, vp, vp, sz, i32],
        "dzs_accel": [vp, i32, vp], "dzs_merge_only": [vp, u64], "dzs_diagnostics": [vp, vp],
        "dzs_get_tables": [vp, vp, vp, vp, vp, vp, vp], "dzs_get_mesh": [vp, i32, vp],
        "dzs_get_counters": [vp, vp], "dzs_get_walk_counters": [vp, vp],
        "dzs_walk_lists": [vp, vp, vp, vp, sz, C.POINTER(sz)],
        "dzs_measure_fp32_peaks": [i32, i32, C.POINTER(C.c_double), C.POINTER(C.c_double)],
        "dzs_debug_fail_alloc": [i32],
        "dzs_batch_create": [vp, i32, i32, C.POINTER(vp)], "dzs_batch_step": [vp, i32, i32, vp],
        "dzs_batch_synchronize": [vp], "dzs_batch_destroy": [vp],
        "dzs_twin_displacement": [vp, vp, vp, i32, vp, vp, C.POINTER(C.c_double)], "dzs_set_profiling": [vp, i32], "dzs_get_profile": [vp, vp, vp],
        "dzs_checkpoint_bytes": [vp, C.POINTER(sz)], "dzs_checkpoint": [vp, vp, sz, C.POINTER(sz)],
        "dzs_restore": [vp, vp, sz],
        "dzs_step_until": [vp, i32, C.POINTER(Halt), C.POINTER(i32), C.POINTER(i32), C.POINTER(C.c_double)],
        "dzs_observe_enable": [vp, C.POINTER(Observe)], "dzs_observe_add_records": [vp, vp, sz],
        "dzs_skymap_get": [vp, vp, sz], "dzs_lcdensity_get": [vp, vp, sz],
        "dzs_skymap_alm": [vp, i32, vp, vp], "dzs_power_spectrum": [vp, i32, i32, vp, vp, vp],
        "dzs_serve": [C.POINTER(ServeConfig), vp, sz, vp, C.POINTER(C.c_double)],
        "dzs_fof": [vp, C.c_double, i32, vp, sz, C.POINTER(sz), vp],
    }
    for name, args in sig.items():
        f = getattr(L, name)
        f.argtypes = args
        f.restype = C.c_int
    L.dzs_morton_sort_noalloc.argtypes = [vp, sz, vp, vp, vp]
    L.dzs_morton_sort_noalloc.restype = C.c_int
    L.dzs_debug_fail_alloc.restype = None
    L.dzs_last_error.argtypes = [vp]
    L.dzs_last_error.restype = C.c_char_p
    _lib = L
    return L


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _check(status, ctx):
    if status != DZS_OK:
        msg = load().dzs_last_error(ctx)
        raise DzsError(status, msg.decode() if msg else "")


def params(**kw) -> Params:
    p = Params()
    load().dzs_params_default(C.byref(p))
    for k, v in kw.items():
        if not hasattr(p, k):
            raise KeyError(k)
        setattr(p, k, v)
    return p


def dzs_footprint_bytes(p: Params) -> int:
    out = C.c_size_t(0)
    _check(load().dzs_footprint_bytes(C.byref(p), C.byref(out)), None)
    return out.value


def dzs_create(p: Params, stream: int = 0):
    h = C.c_void_p()
    _check(load().dzs_create(C.byref(p), C.c_void_p(stream), C.byref(h)), None)
    return h


def dzs_destroy(h):
    load().dzs_destroy(h)


def dzs_ics(h):
    _check(load().dzs_ics(h), h)


def dzs_step(h, n: int) -> int:
    done = C.c_int32(0)
    _check(load().dzs_step(h, n, C.byref(done)), h)
    return done.value


def dzs_run_stages(h, mask: int):
    _check(load().dzs_run_stages(h, mask), h)


def dzs_get_count(h):
    n = C.c_size_t(0)
    st = C.c_int32(0)
    _check(load().dzs_get_count(h, C.byref(n), C.byref(st)), h)
    return n.value, st.value


def dzs_lightcone_drain(h, cap: int = 1 << 22, buf=None):
    """records drained (at most cap), copied out of `buf` (reused when given
    and large enough)"""
    if buf is None or len(buf) < cap:
        buf = np.empty(cap, RECORD_DTYPE)
    n = C.c_size_t(0)
    _check(load().dzs_lightcone_drain(h, _ptr(buf), cap, C.byref(n)), h)
    return buf[:n.value].copy()


def dzs_pipeline(h, on: bool = True):
    _check(load().dzs_pipeline(h, 1 if on else 0), h)


def dzs_step_result(h, step: int):
    """(diagnostics[8], lightcone records written up to that step) of a kept step"""
    out = np.zeros(8)
    w = C.c_uint64(0)
    _check(load().dzs_step_result(h, int(step), _ptr(out), C.byref(w)), h)
    return out, int(w.value)


def dzs_lightcone_drain_step(h, step: int, cap: int = 1 << 22, buf=None):
    """records of the kept steps up to `step` not yet drained (at most cap)"""
    if buf is None or len(buf) < cap:
        buf = np.empty(cap, RECORD_DTYPE)
    n = C.c_size_t(0)
    _check(load().dzs_lightcone_drain_step(h, int(step), _ptr(buf), cap, C.byref(n)), h)
    return buf[:n.value].copy()


def dzs_get_state(h, cap: int = None):
    n, _ = dzs_get_count(h)
    u = np.zeros(3 * n, np.uint32)
    p = np.zeros(3 * n)
    g = np.zeros(3 * n)
    k = np.zeros(n, np.uint32)
    i = np.zeros(n, np.uint32)
    fl = np.zeros(n, np.uint8)
    nn = C.c_size_t(0)
    _check(load().dzs_get_state(h, _ptr(u), _ptr(p), _ptr(g), _ptr(k), _ptr(i), _ptr(fl), n, C.byref(nn)), h)
    return dict(u=u.reshape(3, n), p=p.reshape(3, n), g=g.reshape(3, n), k=k, id=i, fl=fl)


def dzs_set_state(h, state: dict, step: int, with_g: bool = True):
    u = np.ascontiguousarray(state["u"], np.uint32)
    n = u.shape[1]
    p = np.ascontiguousarray(state["p"], np.float64)
    g = np.ascontiguousarray(state["g"], np.float64) if (with_g and "g" in state) else None
    k = np.ascontiguousarray(state["k"], np.uint32)
    i = np.ascontiguousarray(state["id"], np.uint32)
    fl = np.ascontiguousarray(state["fl"], np.uint8)
    _check(load().dzs_set_state(h, _ptr(u), _ptr(p), _ptr(g), _ptr(k), _ptr(i), _ptr(fl), n, step), h)


def dzs_accel(h, parts: int = ACC_ALL):
    n, _ = dzs_get_count(h)
    g = np.zeros(3 * n)
    _check(load().dzs_accel(h, parts, _ptr(g)), h)
    return g.reshape(3, n)


def dzs_merge_only(h, rlat: int):
    _check(load().dzs_merge_only(h, int(rlat)), h)


def dzs_diagnostics(h):
    out = np.zeros(8)
    _check(load().dzs_diagnostics(h, _ptr(out)), h)
    return out


def dzs_get_tables(h, nsteps: int):
    a = np.zeros(nsteps + 1); dr = np.zeros(nsteps); k1 = np.zeros(nsteps); k2 = np.zeros(nsteps)
    rlc = np.zeros(nsteps + 1); rlat = np.zeros(nsteps + 1, np.uint64)
    _check(load().dzs_get_tables(h, _ptr(a), _ptr(dr), _ptr(k1), _ptr(k2), _ptr(rlc), _ptr(rlat)), h)
    return dict(a=a, drift=dr, kick1=k1, kick2=k2, rlc=rlc, rlat=rlat)


def dzs_get_mesh(h, which: int, mesh: int):
    out = np.zeros(mesh ** 3)
    _check(load().dzs_get_mesh(h, which, _ptr(out)), h)
    return out.reshape(mesh, mesh, mesh)


PROFILE_STAGES, PROFILE_WALK = 1, 2


def dzs_set_profiling(h, enable: bool, walk_diag: bool = False):
    """stage timers on/off; walk_diag: also count the walk's node tests,
    rounds and deepest stack use"""
    _check(load().dzs_set_profiling(h, (PROFILE_STAGES if enable else 0) | (PROFILE_WALK if walk_diag else 0)), h)


def dzs_get_profile(h):
    ms = np.zeros(len(PROF_NAMES))
    calls = np.zeros(len(PROF_NAMES), np.uint64)
    _check(load().dzs_get_profile(h, _ptr(ms), _ptr(calls)), h)
    return {name: (float(ms[i]), int(calls[i])) for i, name in enumerate(PROF_NAMES)}


def dzs_get_counters(h):
    out = np.zeros(9, np.uint64)
    _check(load().dzs_get_counters(h, _ptr(out)), h)
    return out


def dzs_get_walk_counters(h):
    """[listed pairs, in-range pairs, node tests, traversal rounds, group walks
    started from the deep frontier window, fallbacks to the shallow frontier]"""
    out = np.zeros(6, np.uint64)
    _check(load().dzs_get_walk_counters(h, _ptr(out)), h)
    return out


def dzs_measure_fp32_peaks(device=0, reps=5):
    """(FP32 FMA TFLOP/s, SFU Gop/s) measured on `device`"""
    f, s = C.c_double(0), C.c_double(0)
    st = load().dzs_measure_fp32_peaks(device, reps, C.byref(f), C.byref(s))
    if st != DZS_OK:
        raise RuntimeError("dzs_measure_fp32_peaks failed with status %d" % st)
    return f.value, s.value


class Batch:
    """Several contexts stepped together by host worker threads (dzs_batch_*);
    the contexts stay the caller's."""

    def __init__(self, contexts, host_threads=0):
        self.contexts = list(contexts)
        arr = (C.c_void_p * max(1, len(self.contexts)))(*[c.h for c in self.contexts])
        h = C.c_void_p()
        st = load().dzs_batch_create(arr, len(self.contexts), host_threads, C.byref(h))
        if st != DZS_OK:
            raise DzsError(st, "dzs_batch_create")
        self.h = h

    def step(self, nsteps, slice=8):
        done = np.zeros(max(1, len(self.contexts)), np.int32)
        st = load().dzs_batch_step(self.h, nsteps, slice, _ptr(done))
        if st != DZS_OK:
            raise DzsError(st, "dzs_batch_step")
        return done[:len(self.contexts)]

    def synchronize(self):
        st = load().dzs_batch_synchronize(self.h)
        if st != DZS_OK:
            raise DzsError(st, "dzs_batch_synchronize")

    def close(self):
        if self.h:
            load().dzs_batch_destroy(self.h)
            self.h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def dzs_debug_fail_alloc(k):
    """test hook: the k-th device allocation from now on fails (0: off)"""
    load().dzs_debug_fail_alloc(int(k))


def dzs_twin_displacement(ha, hb, edges):
    """counts per bin of dx / h (edges in units of h), matched pairs, largest
    dx / h, of the uncrossed twin particles of two contexts"""
    edges = np.ascontiguousarray(edges, np.float64)
    nb = len(edges) - 1
    counts = np.zeros(nb, np.uint64)
    matched = np.zeros(1, np.uint64)
    mx = C.c_double(0)
    _check(load().dzs_twin_displacement(ha, hb, _ptr(edges), nb, _ptr(counts), _ptr(matched), C.byref(mx)), ha)
    return counts, int(matched[0]), mx.value


def dzs_walk_lists(h):
    """per walk group of the last walk: (first particle, count, list length)"""
    ng = C.c_size_t(0)
    _check(load().dzs_walk_lists(h, None, None, None, 0, C.byref(ng)), h)
    n = ng.value
    first = np.zeros(n, np.int64); cnt = np.zeros(n, np.int64); ln = np.zeros(n, np.int64)
    _check(load().dzs_walk_lists(h, _ptr(first), _ptr(cnt), _ptr(ln), n, C.byref(ng)), h)
    return first, cnt, ln


def dzs_morton_sort_noalloc(d_u: int, n: int, d_perm: int, d_keys: int = 0, stream: int = 0) -> int:
    """Allocation-free Morton sort on caller-owned device buffers (raw device
    addresses, e.g. torch tensor data_ptr()); returns the dzs_status code.
    For callers that cannot allocate device memory; see include/dzs.h."""
    return load().dzs_morton_sort_noalloc(C.c_void_p(d_u), n, C.c_void_p(d_perm),
                                          C.c_void_p(d_keys) if d_keys else None, C.c_void_p(stream))


def dzs_checkpoint(h) -> bytes:
    nb = C.c_size_t(0)
    _check(load().dzs_checkpoint_bytes(h, C.byref(nb)), h)
    buf = np.zeros(nb.value, np.uint8)
    w = C.c_size_t(0)
    _check(load().dzs_checkpoint(h, _ptr(buf), nb.value, C.byref(w)), h)
    return buf[:w.value].tobytes()


def dzs_restore(h, blob: bytes):
    buf = np.frombuffer(blob, np.uint8)
    _check(load().dzs_restore(h, _ptr(buf), len(buf)), h)


def dzs_observe_enable(h, nside=0, mesh=0, a_lo=0.0, a_hi=2.0):
    o = Observe(nside, mesh, a_lo, a_hi)
    _check(load().dzs_observe_enable(h, C.byref(o)), h)


def dzs_observe_add_records(h, rec):
    rec = np.ascontiguousarray(rec, RECORD_DTYPE)
    _check(load().dzs_observe_add_records(h, rec.ctypes.data_as(C.c_void_p), len(rec)), h)


def dzs_skymap_get(h, nside):
    m = np.zeros(12 * nside * nside, np.uint64)
    _check(load().dzs_skymap_get(h, _ptr(m), m.size), h)
    return m


def dzs_lcdensity_get(h, mesh):
    g = np.zeros(mesh ** 3, np.uint64)
    _check(load().dzs_lcdensity_get(h, _ptr(g), g.size), h)
    return g.reshape(mesh, mesh, mesh)


def dzs_skymap_alm(h, lmax):
    """-> (C_l [lmax + 1], a_lm [lmax + 1, lmax + 1] complex indexed [l, m])"""
    cl = np.zeros(lmax + 1)
    raw = np.zeros(2 * (lmax + 1) * (lmax + 2) // 2)
    _check(load().dzs_skymap_alm(h, lmax, _ptr(cl), _ptr(raw)), h)
    a = np.zeros((lmax + 1, lmax + 1), np.complex128)
    z = raw[0::2] + 1j * raw[1::2]
    for m in range(lmax + 1):
        i0 = m * (2 * lmax + 1 - m) // 2
        a[m:, m] = z[i0 + m:i0 + lmax + 1]
    return cl, a


def dzs_power_spectrum(h, nbins, shot=True):
    """-> (k [h/Mpc], P(k) [(Mpc/h)^3], modes) per bin"""
    k, p, n = np.zeros(nbins), np.zeros(nbins), np.zeros(nbins)
    _check(load().dzs_power_spectrum(h, nbins, PK_SHOT if shot else 0, _ptr(k), _ptr(p), _ptr(n)), h)
    return k, p, n


def dzs_serve(requests, hbm_budget_bytes, max_active=0, steps_per_slice=8, host_threads=0, **base):
    """requests: iterable of dicts (arrival_s, n1d, mesh, box, sigma8, seed).
    -> (status, wall seconds, list of result dicts with arrival_s and latency_s)"""
    reqs = list(requests)
    arr = (Request * max(1, len(reqs)))()
    for i, r in enumerate(reqs):
        arr[i] = Request(float(r["arrival_s"]), int(r["n1d"]), int(r["mesh"]), float(r["box"]),
                         float(r["sigma8"]), int(r["seed"]))
    res = (RequestResult * max(1, len(reqs)))()
    cfg = ServeConfig(float(hbm_budget_bytes), int(max_active), int(steps_per_slice), int(host_threads), 0,
                      params(**base))
    wall = C.c_double(0)
    st = load().dzs_serve(C.byref(cfg), C.cast(arr, C.c_void_p), len(reqs), C.cast(res, C.c_void_p),
                          C.byref(wall))
    out = []
    for i, r in enumerate(reqs):
        x = res[i]
        out.append(dict(arrival_s=float(r["arrival_s"]), admit_s=x.admit_s, done_s=x.done_s,
                        latency_s=x.done_s - float(r["arrival_s"]), n_end=x.n_end, records=x.records,
                        record_hash=x.record_hash, diag=list(x.diag), status=x.status))
    return st, wall.value, out


def dzs_fof(h, link=0.2, nmin=20, labels=False):
    """-> haloes [HALO_DTYPE] (and per-particle labels when asked)"""
    nh = C.c_size_t(0)
    _check(load().dzs_fof(h, float(link), int(nmin), None, 0, C.byref(nh), None), h)
    n, _ = dzs_get_count(h)
    out = np.zeros(max(1, nh.value), HALO_DTYPE)
    lab = np.zeros(max(1, n), np.int64) if labels else None
    _check(load().dzs_fof(h, float(link), int(nmin), out.ctypes.data_as(C.c_void_p), nh.value, C.byref(nh),
                          _ptr(lab)), h)
    out = out[:nh.value]
    return (out, lab[:n]) if labels else out


def dzs_step_until(h, max_steps: int, ratio_min=0.0, wall_limit_s=0.0, horizon_s=0.0):
    """-> (steps done, DZS_HALT_* reason, last N / N0)"""
    hp = Halt(ratio_min, wall_limit_s, horizon_s)
    done, why, r = C.c_int32(0), C.c_int32(0), C.c_double(0)
    _check(load().dzs_step_until(h, max_steps, C.byref(hp), C.byref(done), C.byref(why), C.byref(r)), h)
    return done.value, why.value, r.value


class Context:
    """Owns one dzs_ctx; methods mirror the C entry points."""

    def __init__(self, p: Params = None, stream: int = 0, **kw):
        self.params = p if p is not None else params(**kw)
        self.h = dzs_create(self.params, stream)

    def close(self):
        if self.h:
            dzs_destroy(self.h)
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

    def ics(self): dzs_ics(self.h)
    def step(self, n=1): return dzs_step(self.h, n)
    def run_stages(self, mask): dzs_run_stages(self.h, mask)
    def count(self): return dzs_get_count(self.h)
    def drain(self, cap=1 << 22):
        if getattr(self, "_drain_buf", None) is None or len(self._drain_buf) < cap:
            self._drain_buf = np.empty(cap, RECORD_DTYPE)
        return dzs_lightcone_drain(self.h, cap, self._drain_buf)
    def pipeline(self, on=True): dzs_pipeline(self.h, on)
    def step_result(self, step): return dzs_step_result(self.h, step)
    def drain_step(self, step, cap=1 << 22, buf=None):
        if buf is None:
            if getattr(self, "_drain_buf", None) is None or len(self._drain_buf) < cap:
                self._drain_buf = np.empty(cap, RECORD_DTYPE)
            buf = self._drain_buf
        return dzs_lightcone_drain_step(self.h, step, cap, buf)
    def state(self): return dzs_get_state(self.h)
    def set_state(self, st, step, with_g=True): dzs_set_state(self.h, st, step, with_g)
    def accel(self, parts=ACC_ALL): return dzs_accel(self.h, parts)
    def merge_only(self, rlat): dzs_merge_only(self.h, rlat)
    def diagnostics(self): return dzs_diagnostics(self.h)
    def tables(self): return dzs_get_tables(self.h, self.params.nsteps)
    def mesh(self, which): return dzs_get_mesh(self.h, which, self.params.mesh)
    def counters(self): return dzs_get_counters(self.h)
    def walk_counters(self): return dzs_get_walk_counters(self.h)
    def walk_lists(self): return dzs_walk_lists(self.h)
    def set_profiling(self, on=True, walk_diag=False): dzs_set_profiling(self.h, on, walk_diag)
    def profile(self): return dzs_get_profile(self.h)
    def checkpoint(self): return dzs_checkpoint(self.h)
    def restore(self, blob): dzs_restore(self.h, blob)
    def step_until(self, max_steps, **halt): return dzs_step_until(self.h, max_steps, **halt)
    def observe(self, **kw): dzs_observe_enable(self.h, **kw)
    def observe_add_records(self, rec): dzs_observe_add_records(self.h, rec)
    def skymap(self, nside): return dzs_skymap_get(self.h, nside)
    def lcdensity(self, mesh): return dzs_lcdensity_get(self.h, mesh)
    def skymap_alm(self, lmax): return dzs_skymap_alm(self.h, lmax)
    def power_spectrum(self, nbins, shot=True): return dzs_power_spectrum(self.h, nbins, shot)
    def fof(self, link=0.2, nmin=20, labels=False): return dzs_fof(self.h, link, nmin, labels)
