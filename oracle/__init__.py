"""FP64 CPU oracle for the ESES hot path -- test infrastructure only.

Only the tests, the package smoke check and the benchmark's CPU-baseline leg
use this package.  It is a plain C implementation of the SES definitions
(§1, Eq. 1-4, Algorithm 1, §2.3-2.5), built with gcc and loaded through
ctypes; it shares no code with the CUDA library.

Functions mirror the C entry points in ``eses_oracle.c``:

* :func:`grid`            -- Eq. 2 grid origin and dimensions;
* :func:`block_count`     -- blocks per axis for B-point blocks with shared faces;
* :func:`run`             -- Algorithm 1 over all blocks (or a sample of them):
  labels, per-axis intersections (lower index, tau, normal, patch type), area,
  volume;
* :func:`distance`        -- min(cap, dist(x, Omega_free)) with its witness;
* :func:`label_points`    -- Eq. 2 labels of arbitrary points;
* :func:`model_stats`     -- number of circle pairs and free triple points.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "eses_oracle.c")
_LIB = os.path.join(_HERE, "_eses_oracle.so")
_lock = threading.Lock()
_lib = None

TYPE_NONE, TYPE_F, TYPE_E, TYPE_V, TYPE_FREE = -1, 0, 1, 2, 3


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain IEEE arithmetic, no contraction)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
           "-std=c11", "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB)
        P = ctypes.c_void_p
        i64 = ctypes.c_int64
        d = ctypes.c_double
        lib.eo_grid.argtypes = [P, P, i64, d, d, P, P]
        lib.eo_grid.restype = ctypes.c_int
        lib.eo_block_count.argtypes = [i64, i64]
        lib.eo_block_count.restype = i64
        lib.eo_run.argtypes = [P, P, i64, d, d, d, i64, ctypes.c_int, ctypes.c_int, ctypes.c_int, P, i64]
        lib.eo_run.restype = P
        lib.eo_result_grid.argtypes = [P, P, P]
        lib.eo_result_labels.argtypes = [P, P]
        lib.eo_result_num_intersections.argtypes = [P, ctypes.c_int]
        lib.eo_result_num_intersections.restype = i64
        lib.eo_result_intersections.argtypes = [P, ctypes.c_int, P, P, P, P]
        lib.eo_result_intersection_atoms.argtypes = [P, ctypes.c_int, P]
        lib.eo_result_stats.argtypes = [P, P]
        lib.eo_result_free.argtypes = [P]
        lib.eo_distance_points.argtypes = [P, P, i64, d, P, i64, d, ctypes.c_int, P, P, P, P, P]
        lib.eo_distance_points.restype = ctypes.c_int
        lib.eo_label_points.argtypes = [P, P, i64, d, P, i64, ctypes.c_int, P]
        lib.eo_label_points.restype = ctypes.c_int
        lib.eo_model_stats.argtypes = [P, P, i64, d, P, P, P, i64, P, i64]
        lib.eo_model_stats.restype = ctypes.c_int
        lib.eo_num_threads.restype = ctypes.c_int
        lib.eo_run_sparse.argtypes = [P, P, i64, d, d, d, i64, ctypes.c_int, P, i64]
        lib.eo_run_grid.argtypes = [P, P, P, i64, d, d, P, P, i64, ctypes.c_int]
        lib.eo_run_grid.restype = P
        lib.eo_run_sparse.restype = ctypes.c_void_p
        lib.eo_result_block_region.argtypes = [ctypes.c_void_p, i64, P, P]
        lib.eo_result_block_region.restype = i64
        lib.eo_result_block_labels.argtypes = [ctypes.c_void_p, i64, P]
        lib.eo_flop_counts.argtypes = [P, P, i64, d, d, d, ctypes.c_int, P]
        lib.eo_flop_counts.restype = ctypes.c_int
        lib.eo_edge_flop_counts.argtypes = [P, P, i64, d, d, d, P, P, ctypes.c_int, P]
        lib.eo_edge_flop_counts.restype = ctypes.c_int
        lib.eo_exterior_labels.argtypes = [P, P]
        lib.eo_exterior_labels.restype = i64
        lib.eo_result_exterior.argtypes = [P]
        lib.eo_result_exterior.restype = i64
        _lib = lib
        return lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _atoms(xyz, radii):
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    radii = np.ascontiguousarray(radii, dtype=np.float64).reshape(-1)
    if xyz.shape[0] != radii.shape[0]:
        raise ValueError("xyz and radii disagree in length")
    return xyz, radii


def num_threads() -> int:
    return int(_load().eo_num_threads())


def grid(xyz, radii, h: float, margin: float):
    """Eq. 2 grid: returns (dims int64[3], lo float64[3])."""
    lib = _load()
    xyz, radii = _atoms(xyz, radii)
    dims = np.zeros(3, np.int64)
    lo = np.zeros(3, np.float64)
    rc = lib.eo_grid(_ptr(xyz), _ptr(radii), xyz.shape[0], h, margin, _ptr(dims), _ptr(lo))
    if rc != 0:
        raise ValueError("invalid grid parameters")
    return dims, lo


def block_count(n_points: int, block_pts: int) -> int:
    return int(_load().eo_block_count(int(n_points), int(block_pts)))


@dataclass
class Result:
    dims: np.ndarray
    lo: np.ndarray
    h: float
    labels: np.ndarray              # int8, dims, C order; -1 where not computed
    idx: list                       # per axis: int64 lower-point linear index
    tau: list                       # per axis: float64 in [0,1]
    normal: list                    # per axis: float64 (n,3), unit, into the solvent
    ptype: list                     # per axis: int32 patch type of the witness
    atoms: list                     # per axis: int64 (n,3) input ids of the witness patch's atoms, -1 padded
    area: float
    volume: float                   # inside length along grid lines (mean of 3 axes)
    volume_count: float             # h^3 * number of inside points
    near_ties: int
    slow_edges: int
    n_points: int


def run(xyz, radii, r_p: float, h: float, margin: float, block_pts: int = 0, nthreads: int = 0,
        brute: bool = False, block_ids=None, exterior: bool = False) -> Result:
    """Algorithm 1 over every block (or the blocks listed in block_ids);
    exterior: the exterior-only surface (cavities filled, reading X1; whole
    grid only)."""
    lib = _load()
    xyz, radii = _atoms(xyz, radii)
    ids = None
    nids = 0
    if block_ids is not None:
        ids = np.ascontiguousarray(block_ids, dtype=np.int64)
        nids = ids.shape[0]
    res = lib.eo_run(_ptr(xyz), _ptr(radii), xyz.shape[0], r_p, h, margin, int(block_pts), int(nthreads),
                     1 if brute else 0, 0, _ptr(ids) if ids is not None else None, nids)
    if not res:
        raise ValueError("invalid parameters")
    return _result(lib, res, h, exterior, block_ids is not None)


def run_on_grid(xyz, radii, r_p: float, h: float, origin, dims, ids=None, block_pts: int = 0,
                nthreads: int = 0) -> Result:
    """Algorithm 1 on a caller-given grid (origin, dims) for atoms carrying
    the caller's ids (reported as the patch atoms; default 0..n-1)."""
    lib = _load()
    xyz, radii = _atoms(xyz, radii)
    o = np.ascontiguousarray(origin, dtype=np.float64).reshape(3)
    dm = np.ascontiguousarray(dims, dtype=np.int64).reshape(3)
    gid = None if ids is None else np.ascontiguousarray(ids, dtype=np.int64).reshape(-1)
    res = lib.eo_run_grid(_ptr(xyz), _ptr(radii), _ptr(gid) if gid is not None else None, xyz.shape[0], r_p, h,
                          _ptr(o), _ptr(dm), int(block_pts), int(nthreads))
    if not res:
        raise ValueError("invalid parameters")
    return _result(lib, res, h, False, False)


def _result(lib, res, h, exterior, sampled) -> Result:
    try:
        if exterior and (sampled or lib.eo_result_exterior(res) < 0):
            raise ValueError("the exterior-only surface needs the whole grid")
        dims = np.zeros(3, np.int64)
        lo = np.zeros(3, np.float64)
        lib.eo_result_grid(res, _ptr(dims), _ptr(lo))
        labels = np.empty(tuple(int(v) for v in dims), np.int8)
        lib.eo_result_labels(res, _ptr(labels))
        idx, tau, nrm, pt, at = [], [], [], [], []
        for a in range(3):
            ne = int(lib.eo_result_num_intersections(res, a))
            i = np.empty(ne, np.int64)
            t = np.empty(ne, np.float64)
            nn = np.empty((ne, 3), np.float64)
            p = np.empty(ne, np.int32)
            w = np.empty((ne, 3), np.int64)
            if ne:
                lib.eo_result_intersections(res, a, _ptr(i), _ptr(t), _ptr(nn), _ptr(p))
                lib.eo_result_intersection_atoms(res, a, _ptr(w))
            idx.append(i); tau.append(t); nrm.append(nn); pt.append(p); at.append(w)
        st = np.zeros(16, np.float64)
        lib.eo_result_stats(res, _ptr(st))
    finally:
        lib.eo_result_free(res)
    return Result(dims=dims, lo=lo, h=h, labels=labels, idx=idx, tau=tau, normal=nrm, ptype=pt, atoms=at,
                  area=float(st[0]), volume=float(st[1]), volume_count=float(st[2]),
                  near_ties=int(st[3]), slow_edges=int(st[4]), n_points=int(st[11]))


def exterior_labels(labels) -> tuple:
    """Flood fill of reading X1 on a label grid (int8, C order): returns
    (labels with cavity points relabelled inside, number relabelled)."""
    lib = _load()
    lab = np.ascontiguousarray(labels, dtype=np.int8).copy()
    dims = np.array(lab.shape, np.int64)
    n = int(lib.eo_exterior_labels(_ptr(lab), _ptr(dims)))
    return lab, n


def run_blocks(xyz, radii, r_p: float, h: float, margin: float, block_pts: int, block_ids, nthreads: int = 0):
    """Algorithm 1 over the listed blocks only, keeping only their owned
    points' labels: returns (dims, lo, blocks, idx, tau, normal) with blocks a
    list of (own_lo, own_hi, labels of the owned region); idx are global."""
    lib = _load()
    xyz, radii = _atoms(xyz, radii)
    ids = np.ascontiguousarray(block_ids, dtype=np.int64)
    res = lib.eo_run_sparse(_ptr(xyz), _ptr(radii), xyz.shape[0], r_p, h, margin, int(block_pts), int(nthreads),
                            _ptr(ids), ids.shape[0])
    if not res:
        raise ValueError("invalid parameters")
    try:
        dims = np.zeros(3, np.int64)
        lo = np.zeros(3, np.float64)
        lib.eo_result_grid(res, _ptr(dims), _ptr(lo))
        blocks = []
        for t in range(ids.shape[0]):
            blo = np.zeros(3, np.int64)
            bhi = np.zeros(3, np.int64)
            cnt = lib.eo_result_block_region(res, t, _ptr(blo), _ptr(bhi))
            lab = np.empty(tuple(int(v) for v in (bhi - blo)), np.int8)
            assert cnt == lab.size
            lib.eo_result_block_labels(res, t, _ptr(lab))
            blocks.append((blo, bhi, lab))
        idx, tau, nrm = [], [], []
        for a in range(3):
            ne = int(lib.eo_result_num_intersections(res, a))
            i = np.empty(ne, np.int64)
            t_ = np.empty(ne, np.float64)
            nn = np.empty((ne, 3), np.float64)
            if ne:
                lib.eo_result_intersections(res, a, _ptr(i), _ptr(t_), _ptr(nn), None)
            idx.append(i); tau.append(t_); nrm.append(nn)
    finally:
        lib.eo_result_free(res)
    return dims, lo, blocks, idx, tau, nrm


def distance(xyz, radii, r_p: float, pts, cap: float, brute: bool = False):
    """min(cap, dist(x, Omega_free)) for each point, with witness point, type and atom ids."""
    lib = _load()
    xyz, radii = _atoms(xyz, radii)
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
    m = pts.shape[0]
    d = np.empty(m, np.float64)
    q = np.empty((m, 3), np.float64)
    t = np.empty(m, np.int32)
    ids = np.empty((m, 3), np.int64)
    cnt = np.empty((m, 5), np.int64)
    lib.eo_distance_points(_ptr(xyz), _ptr(radii), xyz.shape[0], r_p, _ptr(pts), m, cap, 1 if brute else 0,
                           _ptr(d), _ptr(q), _ptr(t), _ptr(ids), _ptr(cnt))
    return d, q, t, ids


def label_points(xyz, radii, r_p: float, pts, brute: bool = False) -> np.ndarray:
    lib = _load()
    xyz, radii = _atoms(xyz, radii)
    pts = np.ascontiguousarray(pts, dtype=np.float64).reshape(-1, 3)
    out = np.empty(pts.shape[0], np.int8)
    lib.eo_label_points(_ptr(xyz), _ptr(radii), xyz.shape[0], r_p, _ptr(pts), pts.shape[0], 1 if brute else 0,
                        _ptr(out))
    return out


def model_stats(xyz, radii, r_p: float, max_vertices: int = 0, max_pairs: int = 0):
    """Circle pairs and free triple points of the whole molecule.

    Returns (n_pairs, n_free_vertices, vertices (<= max_vertices, 3) or None,
    pairs (<= max_pairs, 2) original atom indices or None)."""
    lib = _load()
    xyz, radii = _atoms(xyz, radii)
    npairs = np.zeros(1, np.int64)
    nverts = np.zeros(1, np.int64)
    buf = np.empty((max(max_vertices, 1), 3), np.float64)
    pbuf = np.empty((max(max_pairs, 1), 2), np.int64)
    lib.eo_model_stats(_ptr(xyz), _ptr(radii), xyz.shape[0], r_p, _ptr(npairs), _ptr(nverts),
                       _ptr(buf) if max_vertices else None, max_vertices, _ptr(pbuf) if max_pairs else None, max_pairs)
    nv = int(nverts[0])
    npr = int(npairs[0])
    verts = buf[: min(nv, max_vertices)] if max_vertices else None
    pairs = pbuf[: min(npr, max_pairs)] if max_pairs else None
    return npr, nv, verts, pairs


FLOP_KEYS = ["points", "sum_reach", "shell_points", "sum_face", "sum_face_x_reach", "sum_arc", "sum_vert",
             "model_flops"]


def flop_counts(xyz, radii, r_p: float, h: float, margin: float, nthreads: int = 0) -> dict:
    """Algorithmic flop model of the classification over the whole grid."""
    lib = _load()
    xyz, radii = _atoms(xyz, radii)
    out = np.zeros(8, np.int64)
    rc = lib.eo_flop_counts(_ptr(xyz), _ptr(radii), xyz.shape[0], r_p, h, margin, int(nthreads), _ptr(out))
    if rc != 0:
        raise ValueError("invalid parameters")
    return dict(zip(FLOP_KEYS, (int(v) for v in out)))


EDGE_FLOP_KEYS = ["edges", "vdw_spheres", "probe_spheres", "tori", "model_flops"]


def edge_flop_counts(xyz, radii, r_p: float, h: float, margin: float, idx, nthreads: int = 0) -> dict:
    """Edge terms of the flop model over the crossing edges idx (3 arrays of lower indices)."""
    lib = _load()
    xyz, radii = _atoms(xyz, radii)
    arrs = [np.ascontiguousarray(a, dtype=np.int64) for a in idx]
    ne = np.array([a.shape[0] for a in arrs], np.int64)
    ptrs = (ctypes.c_void_p * 3)(*[a.ctypes.data for a in arrs])
    out = np.zeros(5, np.int64)
    rc = lib.eo_edge_flop_counts(_ptr(xyz), _ptr(radii), xyz.shape[0], r_p, h, margin, _ptr(ne),
                                 ctypes.cast(ptrs, ctypes.c_void_p), int(nthreads), _ptr(out))
    if rc != 0:
        raise ValueError("invalid parameters")
    return dict(zip(EDGE_FLOP_KEYS, (int(v) for v in out)))
