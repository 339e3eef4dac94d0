"""Seeded synthetic inputs shared by the oracle side and the GPU side.

This module produces input bytes only (random walks, noisy copies of collection
members, uniform picks). It holds none of the search method's arithmetic. Host
and device generators give bit-identical fp32 values (see datagen_core.h).

Workload recipes (sizes and value distributions of the paper's experiments,
Section IV "Datasets"): random-walk collections of length-256 series, and query
sets mixing fresh walks with noisy copies of collection members.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_host = None
_dev = None


def _load_host():
    global _host
    if _host is None:
        if not os.path.exists(_build.HOST_LIB):
            _build.build(device=False)
        lib = ctypes.CDLL(_build.HOST_LIB)
        c_i64, c_u64, c_i32 = ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32
        vp = ctypes.c_void_p
        lib.dg_walks_host.argtypes = [c_u64, c_i64, c_i64, c_i32, vp]
        lib.dg_noisy_copies_host.argtypes = [c_u64, c_u64, vp, vp, c_i64, c_i32, vp]
        lib.dg_pick_host.argtypes = [c_u64, c_i64, c_i64, c_i64, vp]
        lib.dg_philox_host.argtypes = [vp, vp, vp]
        lib.dg_ln_host.argtypes = [ctypes.c_float]
        lib.dg_ln_host.restype = ctypes.c_float
        lib.dg_sincos_2pi_host.argtypes = [ctypes.c_float, vp, vp]
        lib.dg_normals_host.argtypes = [c_u64, ctypes.c_uint32, c_u64, c_i32, vp]
        lib.dg_mixed_host.argtypes = [c_u64, c_i64, c_i64, c_i32, vp]
        lib.dg_mixed_noisy_host.argtypes = [c_u64, c_u64, vp, ctypes.c_float, c_i64, c_i32, vp]
        _host = lib
    return _host


def _load_dev():
    global _dev
    if _dev is None:
        if not os.path.exists(_build.DEV_LIB):
            raise RuntimeError("device generator library missing: run __graft_entry__.build()")
        lib = ctypes.CDLL(_build.DEV_LIB)
        c_i64, c_u64, c_i32, vp = ctypes.c_int64, ctypes.c_uint64, ctypes.c_int32, ctypes.c_void_p
        lib.dg_walks_device.argtypes = [c_u64, c_i64, c_i64, c_i32, vp, vp]
        lib.dg_walks_device.restype = ctypes.c_int
        lib.dg_noisy_copies_device.argtypes = [c_u64, c_u64, vp, vp, c_i64, c_i32, vp, vp]
        lib.dg_noisy_copies_device.restype = ctypes.c_int
        lib.dg_mixed_device.argtypes = [c_u64, c_i64, c_i64, c_i32, vp, vp]
        lib.dg_mixed_device.restype = ctypes.c_int
        _dev = lib
    return _dev


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


# ---------------------------------------------------------------- primitives
def walks(seed, first_id, count, length):
    """Random walks first_id .. first_id+count-1 of collection `seed`: float32 [count, length]."""
    out = np.empty((count, length), dtype=np.float32)
    if count:
        _load_host().dg_walks_host(seed, first_id, count, length, _ptr(out))
    return out


def noisy_copies(data_seed, noise_seed, ids, sigmas, length):
    """walk(data_seed, ids[i]) + sigmas[i] * N(0,1) noise drawn from noise_seed, keyed by i."""
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    sigmas = np.ascontiguousarray(sigmas, dtype=np.float32)
    assert ids.shape == sigmas.shape
    out = np.empty((len(ids), length), dtype=np.float32)
    if len(ids):
        _load_host().dg_noisy_copies_host(data_seed, noise_seed, _ptr(ids), _ptr(sigmas), len(ids), length, _ptr(out))
    return out


def mixed(seed, first_id, count, length):
    """Mixed-shape series (noisy sinusoids and Laplace-step walks with a spike burst)
    first_id .. first_id+count-1 of collection `seed`: float32 [count, length]."""
    out = np.empty((count, length), dtype=np.float32)
    if count:
        _load_host().dg_mixed_host(seed, first_id, count, length, _ptr(out))
    return out


def mixed_noisy(data_seed, noise_seed, ids, sigma, length):
    ids = np.ascontiguousarray(ids, dtype=np.int64)
    out = np.empty((len(ids), length), dtype=np.float32)
    if len(ids):
        _load_host().dg_mixed_noisy_host(data_seed, noise_seed, _ptr(ids), float(sigma), len(ids), length, _ptr(out))
    return out


def pick(seed, first, count, n):
    """Uniform picks in [0, n): draws first .. first+count-1."""
    out = np.empty(count, dtype=np.int64)
    if count:
        _load_host().dg_pick_host(seed, first, count, n, _ptr(out))
    return out


def philox4x32_10(ctr, key):
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    o = np.empty(4, dtype=np.uint32)
    _load_host().dg_philox_host(_ptr(c), _ptr(k), _ptr(o))
    return o


def ln(x):
    return _load_host().dg_ln_host(float(x))


def sincos_2pi(u):
    s, c = ctypes.c_float(), ctypes.c_float()
    _load_host().dg_sincos_2pi_host(float(u), ctypes.byref(s), ctypes.byref(c))
    return s.value, c.value


def normals(seed, stream, id_, count):
    out = np.empty(count, dtype=np.float32)
    _load_host().dg_normals_host(seed, stream, id_, count, _ptr(out))
    return out


# ------------------------------------------------------------ device fillers
def walks_device(seed, first_id, count, length, out_ptr, stream_ptr=0):
    """Fill a device buffer (raw pointer) with walks; bit-identical to walks()."""
    rc = _load_dev().dg_walks_device(seed, first_id, count, length, ctypes.c_void_p(out_ptr),
                                     ctypes.c_void_p(stream_ptr))
    if rc != 0:
        raise RuntimeError(f"dg_walks_device failed: cudaError {rc}")


def mixed_device(seed, first_id, count, length, out_ptr, stream_ptr=0):
    """Fill a device buffer (raw pointer) with the mixed-shape family; bit-identical to mixed()."""
    rc = _load_dev().dg_mixed_device(seed, first_id, count, length, ctypes.c_void_p(out_ptr),
                                     ctypes.c_void_p(stream_ptr))
    if rc != 0:
        raise RuntimeError(f"dg_mixed_device failed: cudaError {rc}")


def noisy_copies_device(data_seed, noise_seed, ids_ptr, sigma_ptr, count, length, out_ptr, stream_ptr=0):
    rc = _load_dev().dg_noisy_copies_device(data_seed, noise_seed, ctypes.c_void_p(ids_ptr),
                                            ctypes.c_void_p(sigma_ptr), count, length,
                                            ctypes.c_void_p(out_ptr), ctypes.c_void_p(stream_ptr))
    if rc != 0:
        raise RuntimeError(f"dg_noisy_copies_device failed: cudaError {rc}")


# ------------------------------------------------------------ workload recipes
SIGMAS = (0.01, 0.1, 1.0)


def query_plan(n_collection, count=100, fresh_seed=1, pick_seed=2):
    """Query mix of the 100M x 256 workload: the first half fresh random walks
    (collection `fresh_seed`), the second half noisy copies of collection members
    (ids drawn from `pick_seed`) with sigma cycling through 0.01, 0.1, 1.
    Returns (n_fresh, ids, sigmas) for the copy half."""
    n_fresh = count // 2
    n_copy = count - n_fresh
    ids = pick(pick_seed, 0, n_copy, n_collection)
    sigmas = np.array([SIGMAS[i % 3] for i in range(n_copy)], dtype=np.float32)
    return n_fresh, ids, sigmas


def paper_queries(n_collection, length=256, count=100, data_seed=0, fresh_seed=1, pick_seed=2):
    """Host copy of the query mix (float32 [count, length], un-normalised)."""
    n_fresh, ids, sigmas = query_plan(n_collection, count, fresh_seed, pick_seed)
    fresh = walks(fresh_seed, 0, n_fresh, length)
    copies = noisy_copies(data_seed, pick_seed, ids, sigmas, length)
    return np.concatenate([fresh, copies], axis=0)


def mixed_queries(count=100, length=256, query_seed=5, noise_seed=6, sigma=0.31622777):
    """Query set of the mixed-shape workload: fresh draws from the same generator
    (collection `query_seed`) plus N(0, 0.1) noise (sigma = sqrt 0.1)."""
    return mixed_noisy(query_seed, noise_seed, np.arange(count), sigma, length)
