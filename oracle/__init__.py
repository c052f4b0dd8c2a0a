"""ctypes wrapper of the FP64 CPU oracle (oracle/*.c).

TEST INFRASTRUCTURE ONLY: tests/, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may use it.  The
product path (``paper_2005_05328_gb300``) never imports it.

Arrays follow the oracle's conventions: positions ``u`` are uint32 lattice
coordinates in SoA layout ``[3, n]``; momenta / accelerations are float64
``[3, n]``; ``k`` (mass multiplicity) and ``id`` are uint32; ``fl`` uint8.
"""
from __future__ import annotations

import ctypes as C
import os
from ctypes import byref

import numpy as np

from . import build as _build

_lib = None


class Params(C.Structure):
    _fields_ = [
        ("n1d", C.c_int32), ("mesh", C.c_int32), ("box", C.c_double),
        ("omega_m", C.c_double), ("omega_l", C.c_double), ("hubble", C.c_double),
        ("sigma8", C.c_double), ("ns", C.c_double), ("z_init", C.c_double),
        ("nsteps", C.c_int32), ("leaf_bucket", C.c_int32), ("walk_group", C.c_int32),
        ("dzs_on", C.c_int32), ("merge_level", C.c_int32), ("rlc_mode", C.c_int32),
        ("rs_cells", C.c_double), ("rcut_rs", C.c_double), ("theta", C.c_double),
        ("soft_frac", C.c_double), ("theta_dzs", C.c_double), ("buffer_cells", C.c_double),
        ("seed", C.c_uint64), ("criterion", C.c_int32), ("pad_", C.c_int32), ("alpha_dyn", C.c_double),
    ]


class Record(C.Structure):
    _fields_ = [("id", C.c_uint32), ("k", C.c_uint32), ("a_cross", C.c_double),
                ("x", C.c_double * 3), ("p", C.c_double * 3)]


RECORD_DTYPE = np.dtype([("id", "<u4"), ("k", "<u4"), ("a_cross", "<f8"),
                         ("x", "<f8", (3,)), ("p", "<f8", (3,))])
assert RECORD_DTYPE.itemsize == C.sizeof(Record) == 64

FL_CROSSED = 1
FL_MERGED = 2

DEFAULTS = dict(n1d=32, mesh=64, box=64.0, omega_m=0.3, omega_l=0.7, hubble=0.7,
                sigma8=0.8, ns=0.96, z_init=49.0, nsteps=96, leaf_bucket=8,
                walk_group=32, dzs_on=1, merge_level=2, rlc_mode=0, rs_cells=1.25,
                rcut_rs=4.5, theta=0.5, soft_frac=1.0 / 40.0, theta_dzs=0.1,
                buffer_cells=2.0, seed=1, criterion=0, alpha_dyn=0.01)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        _lib = C.CDLL(path)
        _declare(_lib)
    return _lib


def _p(t):
    return C.POINTER(t)


def _declare(L):
    d, i32, i64, u64 = C.c_double, C.c_int32, C.c_int64, C.c_uint64
    vp = C.c_void_p
    P = _p(Params)
    sig = {
        "dzso_hubble_e": (d, [P, d]), "dzso_drift_factor": (d, [P, d, d]),
        "dzso_kick_factor": (d, [P, d, d]), "dzso_chi": (d, [P, d]),
        "dzso_growth": (d, [P, d]), "dzso_growth_rate": (d, [P, d]),
        "dzso_power": (d, [P, d]), "dzso_power_amplitude": (d, [P]),
        "dzso_power_shape": (d, [P, d]), "dzso_sigma_r": (d, [P, d]),
        "dzso_tables": (None, [P, vp, vp, vp, vp, vp, vp]),
        "dzso_fft1": (None, [C.c_int, vp, C.c_int]),
        "dzso_fft3": (None, [C.c_int, C.c_int, C.c_int, vp, C.c_int]),
        "dzso_white_noise": (None, [u64, C.c_int, vp]),
        "dzso_splitmix64_at": (u64, [u64, u64]),
        "dzso_ics": (None, [P, vp, vp, vp, vp, vp]),
        "dzso_morton_key": (u64, [C.c_uint32, C.c_uint32, C.c_uint32]),
        "dzso_sort": (None, [i64, vp, vp, vp]),
        "dzso_cic_delta": (None, [P, i64, vp, vp, vp]),
        "dzso_pm_potential": (None, [P, vp, vp]),
        "dzso_pm_accel": (None, [P, vp, i64, vp, vp, vp, i64]),
        "dzso_tree_accel": (None, [P, i64, vp, vp, vp, vp, i64]),
        "dzso_pair_factor": (d, [P, d, d]),
        "dzso_count_groups": (i64, [P, i64, vp, vp, vp]),
        "dzso_interaction_count": (i64, [P, i64, vp, vp, i64]),
        "dzso_merge": (i64, [P, i64, u64, d, vp, vp, vp, vp, vp]),
        "dzso_amin2": (d, [i64, vp, vp]),
        "dzso_merge_jmin": (i32, [P]),
        "dzso_merge_threshold": (u64, [P, u64, i32]),
        "dzso_accel": (None, [P, i64, vp, vp, vp, i32, vp, i64]),
        "dzso_kick_drift_cross": (i64, [P, i32, i64, vp, vp, vp, vp, vp, vp, vp]),
        "dzso_step": (i64, [P, i32, i64, vp, vp, vp, vp, vp, vp, vp, vp]),
        "dzso_diagnostics": (None, [P, i64, vp, vp, vp, vp]),
        "dzso_initial_flags": (None, [P, i64, vp, vp]),
        "dzso_ang2pix_ring": (i64, [i64, d, d, d]),
        "dzso_pix2ring": (None, [i64, i64, vp, vp, vp, vp]),
        "dzso_pix2vec_ring": (None, [i64, i64, vp]),
        "dzso_ang2pix_ring_many": (None, [i64, i64, vp, vp]),
        "dzso_pix2vec_ring_many": (None, [i64, i64, vp, vp]),
        "dzso_skymap": (None, [P, i64, vp, i64, d, d, vp]),
        "dzso_pix2zphi_ring_many": (None, [i64, i64, vp, vp, vp]),
        "dzso_lcdensity": (None, [P, i64, vp, i64, d, d, vp]),
        "dzso_fof_threshold": (u64, [P, d]),
        "dzso_fof": (i64, [P, i64, vp, vp, d, i32, vp, vp]),
    }
    for name, (res, args) in sig.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args


def params(**kw) -> Params:
    d = dict(DEFAULTS)
    d.update(kw)
    p = Params()
    for k, v in d.items():
        setattr(p, k, v)
    return p


def _ptr(a):
    return a.ctypes.data_as(C.c_void_p) if a is not None else None


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# ---------------- cosmology ----------------

def hubble_e(P, a): return lib().dzso_hubble_e(C.byref(P), a)
def drift_factor(P, a0, a1): return lib().dzso_drift_factor(C.byref(P), a0, a1)
def kick_factor(P, a0, a1): return lib().dzso_kick_factor(C.byref(P), a0, a1)
def chi(P, a): return lib().dzso_chi(C.byref(P), a)
def growth(P, a): return lib().dzso_growth(C.byref(P), a)
def growth_rate(P, a): return lib().dzso_growth_rate(C.byref(P), a)
def power(P, k): return lib().dzso_power(C.byref(P), k)
def sigma_r(P, r): return lib().dzso_sigma_r(C.byref(P), r)


def tables(P):
    n = P.nsteps
    a = np.zeros(n + 1); dr = np.zeros(n); k1 = np.zeros(n); k2 = np.zeros(n)
    rlc = np.zeros(n + 1); rlat = np.zeros(n + 1, np.uint64)
    lib().dzso_tables(C.byref(P), _ptr(a), _ptr(dr), _ptr(k1), _ptr(k2), _ptr(rlc), _ptr(rlat))
    return dict(a=a, drift=dr, kick1=k1, kick2=k2, rlc=rlc, rlat=rlat)


# ---------------- FFT ----------------

def fft1(x, sign=-1):
    x = np.ascontiguousarray(x, dtype=np.complex128).copy()
    lib().dzso_fft1(len(x), _ptr(x), sign)
    return x


def fft3(x, sign=-1):
    x = np.ascontiguousarray(x, dtype=np.complex128).copy()
    n0, n1, n2 = x.shape
    lib().dzso_fft3(n0, n1, n2, _ptr(x), sign)
    return x


# ---------------- ICs ----------------

def splitmix64_at(seed, c): return lib().dzso_splitmix64_at(seed, c)


def white_noise(seed, n1d):
    w = np.zeros(n1d ** 3)
    lib().dzso_white_noise(seed, n1d, _ptr(w))
    return w


def ics(P):
    n = P.n1d ** 3
    u = np.zeros((3, n), np.uint32); p = np.zeros((3, n)); k = np.zeros(n, np.uint32)
    i = np.zeros(n, np.uint32); fl = np.zeros(n, np.uint8)
    lib().dzso_ics(C.byref(P), _ptr(u), _ptr(p), _ptr(k), _ptr(i), _ptr(fl))
    return dict(u=u, p=p, k=k, id=i, fl=fl)


def initial_flags(P, u, fl):
    u = _c(u, np.uint32); fl = _c(fl, np.uint8).copy()
    lib().dzso_initial_flags(C.byref(P), u.shape[1], _ptr(u), _ptr(fl))
    return fl


# ---------------- sort / keys ----------------

def morton_key(x, y, z): return lib().dzso_morton_key(int(x), int(y), int(z))


def sort(u):
    u = _c(u, np.uint32)
    n = u.shape[1]
    key = np.zeros(n, np.uint64); perm = np.zeros(n, np.int64)
    lib().dzso_sort(n, _ptr(u), _ptr(key), _ptr(perm))
    return key, perm


# ---------------- PM ----------------

def cic_delta(P, u, k):
    u = _c(u, np.uint32); k = _c(k, np.uint32)
    d = np.zeros(P.mesh ** 3)
    lib().dzso_cic_delta(C.byref(P), u.shape[1], _ptr(u), _ptr(k), _ptr(d))
    return d.reshape(P.mesh, P.mesh, P.mesh)


def pm_potential(P, delta):
    delta = _c(delta, np.float64)
    phi = np.zeros(P.mesh ** 3)
    lib().dzso_pm_potential(C.byref(P), _ptr(delta), _ptr(phi))
    return phi.reshape(P.mesh, P.mesh, P.mesh)


def pm_accel(P, phi, u, sample=None):
    phi = _c(phi, np.float64); u = _c(u, np.uint32)
    n = u.shape[1]
    g = np.full((3, n), np.nan)
    s = None if sample is None else _c(sample, np.int64)
    lib().dzso_pm_accel(C.byref(P), _ptr(phi), n, _ptr(u), _ptr(g), _ptr(s), 0 if s is None else len(s))
    return g


# ---------------- tree ----------------

def tree_accel(P, u, k, sample=None):
    """Short-range force; u, k must be Morton-sorted."""
    u = _c(u, np.uint32); k = _c(k, np.uint32)
    n = u.shape[1]
    g = np.full((3, n), np.nan)
    s = None if sample is None else _c(sample, np.int64)
    lib().dzso_tree_accel(C.byref(P), n, _ptr(u), _ptr(k), _ptr(g), _ptr(s), 0 if s is None else len(s))
    return g


def pair_factor(P, r, h): return lib().dzso_pair_factor(C.byref(P), r, h)


def groups(P, u):
    u = _c(u, np.uint32)
    n = u.shape[1]
    ng = lib().dzso_count_groups(C.byref(P), n, _ptr(u), None, None)
    st = np.zeros(ng, np.int64); ct = np.zeros(ng, np.int64)
    lib().dzso_count_groups(C.byref(P), n, _ptr(u), _ptr(st), _ptr(ct))
    return st, ct


def interaction_count(P, u, k, group_index=-1):
    u = _c(u, np.uint32); k = _c(k, np.uint32)
    return lib().dzso_interaction_count(C.byref(P), u.shape[1], _ptr(u), _ptr(k), group_index)


# ---------------- merge ----------------

def merge_jmin(P): return lib().dzso_merge_jmin(C.byref(P))
def merge_threshold(P, rlat, level): return lib().dzso_merge_threshold(C.byref(P), int(rlat), level)


def amin2(g, fl):
    g = _c(g, np.float64); fl = _c(fl, np.uint8)
    return lib().dzso_amin2(g.shape[1], _ptr(g), _ptr(fl))


def merge(P, rlat, state, amin2_value=None):
    """DZS merge on a Morton-sorted state dict; returns a new state dict.  The
    dynamical criterion uses amin2_value, else the state's g and flags."""
    n = state["u"].shape[1]
    if amin2_value is None:
        amin2_value = amin2(state["g"], state["fl"]) if "g" in state else float("inf")
    u = _c(state["u"], np.uint32).copy(); p = _c(state["p"], np.float64).copy()
    k = _c(state["k"], np.uint32).copy(); i = _c(state["id"], np.uint32).copy()
    fl = _c(state["fl"], np.uint8).copy()
    m = lib().dzso_merge(C.byref(P), n, int(rlat), float(amin2_value), _ptr(u), _ptr(p), _ptr(k), _ptr(i),
                         _ptr(fl))
    return dict(u=u.reshape(-1)[:3 * m].reshape(3, m).copy(), p=p.reshape(-1)[:3 * m].reshape(3, m).copy(),
                k=k[:m].copy(), id=i[:m].copy(), fl=fl[:m].copy())


# ---------------- step ----------------

def accel(P, u, k, parts=3, sample=None):
    u = _c(u, np.uint32); k = _c(k, np.uint32)
    n = u.shape[1]
    g = np.full((3, n), np.nan)
    s = None if sample is None else _c(sample, np.int64)
    lib().dzso_accel(C.byref(P), n, _ptr(u), _ptr(k), _ptr(g), parts, _ptr(s), 0 if s is None else len(s))
    return g


def kick_drift_cross(P, step, state, g):
    n = state["u"].shape[1]
    st = {key: np.ascontiguousarray(v).copy() for key, v in state.items()}
    g = _c(g, np.float64)
    rec = np.zeros(n, RECORD_DTYPE)
    nr = lib().dzso_kick_drift_cross(C.byref(P), step, n, _ptr(st["u"]), _ptr(st["p"]), _ptr(g),
                                     _ptr(st["k"]), _ptr(st["id"]), _ptr(st["fl"]), _ptr(rec))
    return st, rec[:nr].copy()


def step(P, stepno, state):
    """One KDK step of a state dict with keys u, p, g, k, id, fl; returns
    (new state, records)."""
    n = state["u"].shape[1]
    u = _c(state["u"], np.uint32).copy(); p = _c(state["p"], np.float64).copy()
    g = _c(state["g"], np.float64).copy(); k = _c(state["k"], np.uint32).copy()
    i = _c(state["id"], np.uint32).copy(); fl = _c(state["fl"], np.uint8).copy()
    rec = np.zeros(n, RECORD_DTYPE)
    nrec = C.c_int64(0)
    m = lib().dzso_step(C.byref(P), stepno, n, _ptr(u), _ptr(p), _ptr(g), _ptr(k), _ptr(i),
                        _ptr(fl), _ptr(rec), C.byref(nrec))
    if m < 0:
        raise ValueError("oracle step rejected")

    def cut3(a):
        return a.reshape(-1)[:3 * m].reshape(3, m).copy()
    return (dict(u=cut3(u), p=cut3(p), g=cut3(g), k=k[:m].copy(), id=i[:m].copy(), fl=fl[:m].copy()),
            rec[:nrec.value].copy())


def diagnostics(P, u, p, k):
    u = _c(u, np.uint32); p = _c(p, np.float64); k = _c(k, np.uint32)
    out = np.zeros(8)
    lib().dzso_diagnostics(C.byref(P), u.shape[1], _ptr(u), _ptr(p), _ptr(k), _ptr(out))
    return out


def initial_state(P):
    """ICs with initial flags and the first accelerations, Morton-sorted (the
    state a KDK step starts from)."""
    st = ics(P)
    st["fl"] = initial_flags(P, st["u"], st["fl"])
    key, perm = sort(st["u"])
    st = {"u": st["u"][:, perm].copy(), "p": st["p"][:, perm].copy(), "k": st["k"][perm].copy(),
          "id": st["id"][perm].copy(), "fl": st["fl"][perm].copy()}
    st["g"] = accel(P, st["u"], st["k"])
    return st


# ---------------- lightcone observables ----------------

def ang2pix(nside, v):
    """RING pixel of each direction v [3, n] (need not be unit vectors)"""
    v = _c(np.atleast_2d(np.asarray(v, np.float64).T).T, np.float64)
    if v.ndim == 1:
        v = v.reshape(3, 1)
    n = v.shape[1]
    pix = np.zeros(n, np.int64)
    lib().dzso_ang2pix_ring_many(int(nside), n, _ptr(v), _ptr(pix))
    return pix


def pix2vec(nside, pix):
    pix = _c(np.atleast_1d(pix), np.int64)
    v = np.zeros((3, len(pix)))
    lib().dzso_pix2vec_ring_many(int(nside), len(pix), _ptr(pix), _ptr(v))
    return v


def pix2ring(nside, pix):
    """-> (ring 1..4 nside - 1, position j 1-based, z, phi) of one pixel"""
    r, j, z, ph = C.c_int64(0), C.c_int64(0), C.c_double(0), C.c_double(0)
    lib().dzso_pix2ring(int(nside), int(pix), byref(r), byref(j), byref(z), byref(ph))
    return r.value, j.value, z.value, ph.value


def pix2zphi(nside, pix):
    """centre z = cos(theta) and phi of each pixel"""
    pix = _c(np.atleast_1d(pix), np.int64)
    z, ph = np.zeros(len(pix)), np.zeros(len(pix))
    lib().dzso_pix2zphi_ring_many(int(nside), len(pix), _ptr(pix), _ptr(z), _ptr(ph))
    return z, ph


def skymap(P, rec, nside, a_lo=0.0, a_hi=2.0):
    """mass (sum of k) per RING pixel of the records with a_lo <= a_cross < a_hi"""
    rec = np.ascontiguousarray(rec, RECORD_DTYPE)
    m = np.zeros(12 * nside * nside, np.uint64)
    lib().dzso_skymap(byref(P), len(rec), rec.ctypes.data_as(C.c_void_p), int(nside), float(a_lo),
                      float(a_hi), _ptr(m))
    return m


def lcdensity(P, rec, mesh, a_lo=0.0, a_hi=2.0):
    """NGP mass grid [mesh, mesh, mesh] of the records' crossing positions"""
    rec = np.ascontiguousarray(rec, RECORD_DTYPE)
    g = np.zeros(mesh ** 3, np.uint64)
    lib().dzso_lcdensity(byref(P), len(rec), rec.ctypes.data_as(C.c_void_p), int(mesh), float(a_lo),
                         float(a_hi), _ptr(g))
    return g.reshape(mesh, mesh, mesh)


# ---------------- friends-of-friends ----------------

HALO_DTYPE = np.dtype([("first", "<i8"), ("count", "<i8"), ("mass", "<u8"), ("x", "<f8", (3,)),
                       ("rmax2", "<u8")])


def fof_threshold(P, link): return lib().dzso_fof_threshold(byref(P), float(link))


def fof(P, u, k, link=0.2, nmin=20):
    """-> (haloes [HALO_DTYPE], label per particle: first member or -1)"""
    u = _c(u, np.uint32); k = _c(k, np.uint32)
    n = u.shape[1]
    lab = np.zeros(n, np.int64)
    h = np.zeros(max(n, 1), HALO_DTYPE)
    nh = lib().dzso_fof(byref(P), n, _ptr(u), _ptr(k), float(link), int(nmin), _ptr(lab),
                        h.ctypes.data_as(C.c_void_p))
    return h[:nh].copy(), lab
