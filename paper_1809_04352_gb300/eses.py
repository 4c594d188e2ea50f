"""Thin Python binding of the libeses C ABI (include/eses.h).

Argument marshalling only: every function calls the C entry point of the same
name, and every step of the surface computation runs in the CUDA kernels of
libeses.so.  The library must have been built (``paper_1809_04352_gb300.build``);
loading fails loudly otherwise -- there is no CPU fallback.

Host arrays are numpy arrays; device arrays may be given as raw pointers
(int) or as objects exposing ``data_ptr()`` (torch CUDA tensors).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

ESES_OK = 0
ESES_EINVAL = -1
ESES_ENOMEM = -2
ESES_ECUDA = -3
ESES_ETIMEOUT = -4
ESES_ECAPACITY = -5
ESES_ESTATE = -6
ESES_EROOT = -7

ESES_OPT_BLOCK_PTS = 1
ESES_OPT_PRECISION = 2
ESES_OPT_STREAM = 3
ESES_OPT_SYNC = 4
ESES_OPT_PROFILE = 5
ESES_OPT_GRAPH = 6
ESES_OPT_QUEUE = 7
ESES_OPT_CLS_CTAS = 8
ESES_OPT_CLS_TILES = 9
ESES_OPT_EDGE_CTAS = 10
ESES_OPT_EDGE_TILES = 11
ESES_OPT_ROOT_THREADS = 12
ESES_OPT_EXTERIOR = 13
ESES_OPT_TC_WAIT = 14
ESES_OPT_FAIL_ALLOC = 15
ESES_OPT_CULL = 16

ESES_PROPOSER_OFF = 0
ESES_PROPOSER_MLP = 1
ESES_PROPOSER_CERTIFY = 2
ESES_MLP_NPARAM = 6337

ESES_PREC_FP64 = 0
ESES_PREC_FP32_FILTERED = 1

STAT_NAMES = ["points", "tiles", "work_tiles", "circle_pairs", "free_arc_pairs", "free_vertices", "band_points",
              "crossing_edges", "root_failures", "inside_points", "kernel_launches", "tiles_proposed_far",
              "tiles_certified", "cavity_points", "exterior_sweeps", "big_tier_tiles", "witness_atom_tests",
              "sphere_candidates", "torus_candidates", "hard_edges"]

# every exported C symbol, as declared in include/eses.h
SYMBOLS = ["eses_create", "eses_create_device", "eses_create_batch", "eses_run_batch", "eses_set_option",
           "eses_get_option", "eses_autotune", "eses_run", "eses_num_molecules", "eses_mol_grid", "eses_mol_labels",
           "eses_mol_labels_device", "eses_mol_num_intersections", "eses_mol_intersections",
           "eses_mol_intersections_device", "eses_mol_area_volume", "eses_grid", "eses_labels",
           "eses_labels_device", "eses_num_intersections", "eses_intersections", "eses_intersections_device",
           "eses_area_volume", "eses_stats", "eses_stage_times", "eses_root_failures", "eses_patch_counts",
           "eses_patch_data", "eses_crossing_edges_noalloc", "eses_set_proposer", "eses_num_tiles",
           "eses_tile_data", "eses_mlp_forward", "eses_mlp_forward_tc", "eses_mlp_grad_scratch", "eses_mlp_grad", "eses_mlp_adam",
           "eses_mesh_count", "eses_mesh", "eses_mesh_table", "eses_intersection_patches", "eses_create_on_grid",
           "eses_num_blocks", "eses_set_blocks", "eses_owned_box",
           "eses_mol_intersection_patches", "eses_last_error", "eses_destroy"]
STAGE_NAMES = ["binning", "pairs", "arcs", "classify", "band", "edge_count", "edge_solve", "edge_polish", "reduce"]

_lib = None


class EsesError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"libeses error {code}: {msg}")
        self.code = code


def library_path() -> str:
    return _build.LIB


def load():
    """Load libeses.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build the CUDA library first "
                           "(paper_1809_04352_gb300.build.build())")
    lib = ctypes.CDLL(path)
    P, i64, d, ci = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double, ctypes.c_int
    PP = ctypes.POINTER(ctypes.c_void_p)
    lib.eses_create.argtypes = [P, P, i64, d, d, d, PP]
    lib.eses_create_device.argtypes = [P, P, i64, d, d, d, PP]
    lib.eses_create_batch.argtypes = [P, P, P, ci, d, d, d, PP]
    lib.eses_run_batch.argtypes = [ci, P, P, P, d, d, d, PP]
    lib.eses_get_option.argtypes = [P, ci, P]
    lib.eses_autotune.argtypes = [P, ci, P]
    lib.eses_num_molecules.argtypes = [P, P]
    lib.eses_mol_grid.argtypes = [P, ci, P, P]
    lib.eses_mol_labels.argtypes = [P, ci, P]
    lib.eses_mol_labels_device.argtypes = [P, ci, PP]
    lib.eses_mol_num_intersections.argtypes = [P, ci, ci, P]
    lib.eses_mol_intersections.argtypes = [P, ci, ci, P, P, P, P, P]
    lib.eses_mol_intersections_device.argtypes = [P, ci, ci, PP, PP, PP, PP, PP]
    lib.eses_mol_area_volume.argtypes = [P, ci, P, P]
    lib.eses_set_option.argtypes = [P, ci, i64]
    lib.eses_set_proposer.argtypes = [P, ci, P, d]
    lib.eses_num_tiles.argtypes = [P, P]
    lib.eses_tile_data.argtypes = [P, P, P]
    lib.eses_mlp_forward.argtypes = [P, i64, P, P, P]
    lib.eses_mlp_forward_tc.argtypes = [P, i64, P, P, P, P]
    lib.eses_mlp_grad_scratch.argtypes = [i64]
    lib.eses_mlp_grad.argtypes = [P, P, P, i64, P, P, P, P, P]
    lib.eses_mlp_adam.argtypes = [P, P, P, P, ci, ctypes.c_float, P]
    lib.eses_run.argtypes = [P]
    lib.eses_grid.argtypes = [P, P, P]
    lib.eses_labels.argtypes = [P, P]
    lib.eses_labels_device.argtypes = [P, PP]
    lib.eses_num_intersections.argtypes = [P, ci, P]
    lib.eses_intersections.argtypes = [P, ci, P, P, P, P, P]
    lib.eses_intersections_device.argtypes = [P, ci, PP, PP, PP, PP, PP]
    lib.eses_area_volume.argtypes = [P, P, P]
    lib.eses_stats.argtypes = [P, P, ci]
    lib.eses_stage_times.argtypes = [P, P, ci]
    lib.eses_root_failures.argtypes = [P, P, ci, P]
    lib.eses_patch_counts.argtypes = [P, P, P, P]
    lib.eses_patch_data.argtypes = [P, P, P, P, P]
    lib.eses_crossing_edges_noalloc.argtypes = [P, P, P, P, P, P, P, P]
    lib.eses_intersection_patches.argtypes = [P, ci, P, P]
    lib.eses_create_on_grid.argtypes = [P, P, i64, d, d, P, P, PP]
    lib.eses_num_blocks.argtypes = [P, P]
    lib.eses_set_blocks.argtypes = [P, P, P]
    lib.eses_owned_box.argtypes = [P, P, P]
    lib.eses_mol_intersection_patches.argtypes = [P, ci, ci, P, P]
    lib.eses_mesh_count.argtypes = [P, P]
    lib.eses_mesh.argtypes = [P, P, P]
    lib.eses_mesh_table.argtypes = [P, P]
    lib.eses_last_error.argtypes = [P]
    lib.eses_last_error.restype = ctypes.c_char_p
    lib.eses_destroy.argtypes = [P]
    lib.eses_destroy.restype = None
    for name in SYMBOLS:
        if name not in ("eses_last_error", "eses_destroy"):
            getattr(lib, name).restype = ctypes.c_int
    lib.eses_mlp_grad_scratch.restype = i64
    _lib = lib
    return lib


def _ptr(a):
    if a is None:
        return None
    if isinstance(a, int):
        return ctypes.c_void_p(a)
    if hasattr(a, "data_ptr"):
        return ctypes.c_void_p(a.data_ptr())
    return a.ctypes.data_as(ctypes.c_void_p)


def _check(rc: int, ctx=None):
    if rc != ESES_OK:
        raise EsesError(rc, eses_last_error(ctx))


def eses_last_error(ctx=None) -> str:
    msg = load().eses_last_error(ctx)
    return msg.decode() if msg else ""


def eses_create(xyz, radii, r_p: float, h: float, margin: float):
    """Host atoms (n,3) float64 and radii (n,) float64 -> context handle."""
    lib = load()
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    radii = np.ascontiguousarray(radii, dtype=np.float64).reshape(-1)
    if xyz.shape[0] != radii.shape[0]:
        raise ValueError("xyz and radii disagree in length")
    out = ctypes.c_void_p()
    _check(lib.eses_create(_ptr(xyz), _ptr(radii), xyz.shape[0], r_p, h, margin, ctypes.byref(out)))
    return out


def eses_create_on_grid(xyz, radii, r_p: float, h: float, origin, dims):
    """Host atoms on a caller-given grid (origin float64[3], dims int64[3]) -> context handle."""
    lib = load()
    xyz = np.ascontiguousarray(xyz, dtype=np.float64).reshape(-1, 3)
    radii = np.ascontiguousarray(radii, dtype=np.float64).reshape(-1)
    if xyz.shape[0] != radii.shape[0]:
        raise ValueError("xyz and radii disagree in length")
    o = np.ascontiguousarray(origin, dtype=np.float64).reshape(3)
    dm = np.ascontiguousarray(dims, dtype=np.int64).reshape(3)
    out = ctypes.c_void_p()
    _check(lib.eses_create_on_grid(_ptr(xyz), _ptr(radii), xyz.shape[0], r_p, h, _ptr(o), _ptr(dm),
                                   ctypes.byref(out)))
    return out


def eses_num_blocks(ctx):
    nb = np.zeros(3, np.int64)
    _check(load().eses_num_blocks(ctx, _ptr(nb)), ctx)
    return nb


def eses_set_blocks(ctx, block_lo=None, block_hi=None):
    """Restrict the next runs to blocks [block_lo, block_hi) per axis (None, None: the whole grid)."""
    if block_lo is None:
        _check(load().eses_set_blocks(ctx, None, None), ctx)
        return
    lo = np.ascontiguousarray(block_lo, dtype=np.int64).reshape(3)
    hi = np.ascontiguousarray(block_hi, dtype=np.int64).reshape(3)
    _check(load().eses_set_blocks(ctx, _ptr(lo), _ptr(hi)), ctx)


def eses_owned_box(ctx):
    lo = np.zeros(3, np.int64)
    dims = np.zeros(3, np.int64)
    _check(load().eses_owned_box(ctx, _ptr(lo), _ptr(dims)), ctx)
    return lo, dims


def eses_create_device(xyz, radii, n_atoms: int, r_p: float, h: float, margin: float):
    """Device atoms (pointer or CUDA tensor, n*3 float64) and radii -> context handle."""
    lib = load()
    out = ctypes.c_void_p()
    _check(lib.eses_create_device(_ptr(xyz), _ptr(radii), int(n_atoms), r_p, h, margin, ctypes.byref(out)))
    return out


def _batch_arrays(mols):
    xyz = [np.ascontiguousarray(x, dtype=np.float64).reshape(-1, 3) for x, _ in mols]
    rad = [np.ascontiguousarray(r, dtype=np.float64).reshape(-1) for _, r in mols]
    for x, r in zip(xyz, rad):
        if x.shape[0] != r.shape[0]:
            raise ValueError("xyz and radii disagree in length")
    counts = np.array([x.shape[0] for x in xyz], np.int64)
    return xyz, rad, counts


def eses_create_batch(mols, r_p: float, h: float, margin: float):
    """Molecules [(xyz (n,3), radii (n,)), ...] sharing r_p, h, margin -> context handle."""
    lib = load()
    xyz, rad, counts = _batch_arrays(mols)
    X = np.ascontiguousarray(np.concatenate(xyz, 0))
    R = np.ascontiguousarray(np.concatenate(rad, 0))
    out = ctypes.c_void_p()
    _check(lib.eses_create_batch(_ptr(X), _ptr(R), _ptr(counts), len(xyz), r_p, h, margin, ctypes.byref(out)))
    return out


def eses_run_batch(mols, r_p: float, h: float, margin: float):
    """Create a batch context from per-molecule arrays and run it once."""
    lib = load()
    xyz, rad, counts = _batch_arrays(mols)
    px = (ctypes.c_void_p * len(xyz))(*[x.ctypes.data for x in xyz])
    pr = (ctypes.c_void_p * len(rad))(*[r.ctypes.data for r in rad])
    out = ctypes.c_void_p()
    _check(lib.eses_run_batch(len(xyz), ctypes.cast(px, ctypes.c_void_p), ctypes.cast(pr, ctypes.c_void_p),
                              _ptr(counts), r_p, h, margin, ctypes.byref(out)))
    return out


def eses_set_option(ctx, key: int, value: int):
    _check(load().eses_set_option(ctx, key, int(value)), ctx)


def eses_get_option(ctx, key: int) -> int:
    v = np.zeros(1, np.int64)
    _check(load().eses_get_option(ctx, key, _ptr(v)), ctx)
    return int(v[0])


def eses_autotune(ctx, reps: int = 3):
    """Time the persistent kernels' launch shapes and keep the fastest; returns
    (classification ms, root-solve ms) of the chosen shapes."""
    ms = np.zeros(2, np.float64)
    _check(load().eses_autotune(ctx, int(reps), _ptr(ms)), ctx)
    return float(ms[0]), float(ms[1])


def eses_set_proposer(ctx, mode: int, params=None, p_far: float = 0.5):
    """Tile proposer mode (ESES_PROPOSER_*); params: host float32[ESES_MLP_NPARAM] or None."""
    if params is not None:
        params = np.ascontiguousarray(params, dtype=np.float32).reshape(-1)
        if params.shape[0] != ESES_MLP_NPARAM:
            raise ValueError(f"expected {ESES_MLP_NPARAM} parameters")
    _check(load().eses_set_proposer(ctx, int(mode), _ptr(params), float(p_far)), ctx)


def eses_num_tiles(ctx) -> int:
    n = np.zeros(1, np.int64)
    _check(load().eses_num_tiles(ctx, _ptr(n)), ctx)
    return int(n[0])


def eses_tile_data(ctx, features=None, targets=None):
    """Device outputs (torch CUDA tensors or pointers): features float32[n_tiles, 32], targets uint8[n_tiles]."""
    _check(load().eses_tile_data(ctx, _ptr(features), _ptr(targets)), ctx)


def _stream(stream):
    return ctypes.c_void_p(int(stream)) if stream else None


def eses_mlp_forward(X, n: int, params, z, stream=0):
    _check(load().eses_mlp_forward(_ptr(X), int(n), _ptr(params), _ptr(z), _stream(stream)))


def eses_mlp_forward_tc(X, n: int, params, z, err, stream=0):
    _check(load().eses_mlp_forward_tc(_ptr(X), int(n), _ptr(params), _ptr(z), _ptr(err), _stream(stream)))


def eses_mlp_grad_scratch(n: int) -> int:
    return int(load().eses_mlp_grad_scratch(int(n)))


def eses_mlp_grad(X, y, w, n: int, params, grad, loss, scratch, stream=0):
    _check(load().eses_mlp_grad(_ptr(X), _ptr(y), _ptr(w), int(n), _ptr(params), _ptr(grad), _ptr(loss),
                                _ptr(scratch), _stream(stream)))


def eses_mlp_adam(params, grad, m, v, step: int, lr: float, stream=0):
    _check(load().eses_mlp_adam(_ptr(params), _ptr(grad), _ptr(m), _ptr(v), int(step), ctypes.c_float(lr),
                                _stream(stream)))


def eses_num_molecules(ctx) -> int:
    n = np.zeros(1, np.int32)
    _check(load().eses_num_molecules(ctx, _ptr(n)), ctx)
    return int(n[0])


def eses_mol_grid(ctx, m: int):
    dims = np.zeros(3, np.int64)
    origin = np.zeros(3, np.float64)
    _check(load().eses_mol_grid(ctx, int(m), _ptr(dims), _ptr(origin)), ctx)
    return dims, origin


def eses_mol_labels(ctx, m: int, out=None):
    dims, _ = eses_mol_grid(ctx, m)
    if out is None:
        out = np.empty(tuple(int(v) for v in dims), np.int8)
    _check(load().eses_mol_labels(ctx, int(m), _ptr(out)), ctx)
    return out


def eses_mol_labels_device(ctx, m: int) -> int:
    p = ctypes.c_void_p()
    _check(load().eses_mol_labels_device(ctx, int(m), ctypes.byref(p)), ctx)
    return int(p.value or 0)


def eses_mol_num_intersections(ctx, m: int, axis: int) -> int:
    n = np.zeros(1, np.int64)
    _check(load().eses_mol_num_intersections(ctx, int(m), axis, _ptr(n)), ctx)
    return int(n[0])


def eses_mol_intersections(ctx, m: int, axis: int, fp32: bool = True):
    """Host copies of molecule m's intersections along one axis."""
    n = eses_mol_num_intersections(ctx, m, axis)
    idx = np.empty(n, np.int64)
    tau = np.empty(n, np.float64)
    nrm = np.empty((n, 3), np.float64)
    t32 = np.empty(n, np.float32) if fp32 else None
    n32 = np.empty((n, 3), np.float32) if fp32 else None
    if n:
        _check(load().eses_mol_intersections(ctx, int(m), axis, _ptr(idx), _ptr(tau), _ptr(nrm), _ptr(t32),
                                             _ptr(n32)), ctx)
    out = {"idx": idx, "tau": tau, "normal": nrm}
    if fp32:
        out["tau32"] = t32
        out["normal32"] = n32
    return out


def eses_mol_intersections_device(ctx, m: int, axis: int):
    ps = [ctypes.c_void_p() for _ in range(5)]
    _check(load().eses_mol_intersections_device(ctx, int(m), axis, *[ctypes.byref(p) for p in ps]), ctx)
    return tuple(int(p.value or 0) for p in ps)


def eses_mol_area_volume(ctx, m: int):
    a = np.zeros(1, np.float64)
    v = np.zeros(1, np.float64)
    _check(load().eses_mol_area_volume(ctx, int(m), _ptr(a), _ptr(v)), ctx)
    return float(a[0]), float(v[0])


def eses_run(ctx):
    _check(load().eses_run(ctx), ctx)


def eses_grid(ctx):
    dims = np.zeros(3, np.int64)
    origin = np.zeros(3, np.float64)
    _check(load().eses_grid(ctx, _ptr(dims), _ptr(origin)), ctx)
    return dims, origin


def eses_labels(ctx, out=None):
    """Host copy of the labels: the whole grid, or the owned box of a block selection."""
    _, dims = eses_owned_box(ctx)
    if out is None:
        out = np.empty(tuple(int(v) for v in dims), np.int8)
    _check(load().eses_labels(ctx, _ptr(out)), ctx)
    return out


ESES_MESH_MAXT = 5


def eses_mesh_count(ctx) -> int:
    """Make the triangle mesh of the last run (one molecule); its triangle count."""
    n = np.zeros(1, np.int64)
    _check(load().eses_mesh_count(ctx, _ptr(n)), ctx)
    return int(n[0])


def eses_mesh(ctx):
    """(keys int64 (n, 3), xyz float64 (n, 3, 3)) of the mesh of the last run."""
    n = eses_mesh_count(ctx)
    keys = np.empty((n, 3), np.int64)
    xyz = np.empty((n, 3, 3), np.float64)
    if n:
        _check(load().eses_mesh(ctx, _ptr(keys), _ptr(xyz)), ctx)
    return keys, xyz


def eses_mesh_table():
    """The mesh's 256-case table: (tri int8 (256, ESES_MESH_MAXT, 3), ntri uint8 (256,))."""
    tri = np.empty((256, ESES_MESH_MAXT, 3), np.int8)
    ntri = np.empty(256, np.uint8)
    _check(load().eses_mesh_table(_ptr(tri), _ptr(ntri)))
    return tri, ntri


def eses_labels_device(ctx) -> int:
    p = ctypes.c_void_p()
    _check(load().eses_labels_device(ctx, ctypes.byref(p)), ctx)
    return int(p.value or 0)


def eses_num_intersections(ctx, axis: int) -> int:
    n = np.zeros(1, np.int64)
    _check(load().eses_num_intersections(ctx, axis, _ptr(n)), ctx)
    return int(n[0])


def eses_intersections(ctx, axis: int, fp32: bool = True):
    """Host copies of one axis' intersections: dict of numpy arrays."""
    n = eses_num_intersections(ctx, axis)
    idx = np.empty(n, np.int64)
    tau = np.empty(n, np.float64)
    nrm = np.empty((n, 3), np.float64)
    t32 = np.empty(n, np.float32) if fp32 else None
    n32 = np.empty((n, 3), np.float32) if fp32 else None
    if n:
        _check(load().eses_intersections(ctx, axis, _ptr(idx), _ptr(tau), _ptr(nrm), _ptr(t32), _ptr(n32)), ctx)
    out = {"idx": idx, "tau": tau, "normal": nrm}
    if fp32:
        out["tau32"] = t32
        out["normal32"] = n32
    return out


def eses_intersection_patches(ctx, axis: int):
    """Patch kind (int8 (n,)) and generating input atoms (int32 (n, 3), ascending,
    -1 padded) of one axis' intersections, in the order of eses_intersections."""
    n = eses_num_intersections(ctx, axis)
    kind = np.empty(n, np.int8)
    atoms = np.empty((n, 3), np.int32)
    if n:
        _check(load().eses_intersection_patches(ctx, axis, _ptr(kind), _ptr(atoms)), ctx)
    return kind, atoms


def eses_mol_intersection_patches(ctx, m: int, axis: int):
    n = eses_mol_num_intersections(ctx, m, axis)
    kind = np.empty(n, np.int8)
    atoms = np.empty((n, 3), np.int32)
    if n:
        _check(load().eses_mol_intersection_patches(ctx, int(m), axis, _ptr(kind), _ptr(atoms)), ctx)
    return kind, atoms


def eses_intersections_device(ctx, axis: int):
    ps = [ctypes.c_void_p() for _ in range(5)]
    _check(load().eses_intersections_device(ctx, axis, *[ctypes.byref(p) for p in ps]), ctx)
    return tuple(int(p.value or 0) for p in ps)


def eses_area_volume(ctx):
    a = np.zeros(1, np.float64)
    v = np.zeros(1, np.float64)
    _check(load().eses_area_volume(ctx, _ptr(a), _ptr(v)), ctx)
    return float(a[0]), float(v[0])


def eses_stats(ctx) -> dict:
    out = np.zeros(len(STAT_NAMES), np.int64)
    _check(load().eses_stats(ctx, _ptr(out), len(STAT_NAMES)), ctx)
    return dict(zip(STAT_NAMES, (int(v) for v in out)))


def eses_stage_times(ctx) -> dict:
    out = np.zeros(len(STAGE_NAMES), np.float64)
    _check(load().eses_stage_times(ctx, _ptr(out), len(STAGE_NAMES)), ctx)
    return dict(zip(STAGE_NAMES, (float(v) for v in out)))


def eses_root_failures(ctx):
    recs = np.zeros((8, 24), np.int64)
    n = np.zeros(1, np.int32)
    _check(load().eses_root_failures(ctx, _ptr(recs), 8, _ptr(n)), ctx)
    return recs[: int(n[0])]


def eses_patch_counts(ctx):
    a, b, c = (np.zeros(1, np.int64) for _ in range(3))
    _check(load().eses_patch_counts(ctx, _ptr(a), _ptr(b), _ptr(c)), ctx)
    return int(a[0]), int(b[0]), int(c[0])


def eses_patch_data(ctx):
    np_, _, nv = eses_patch_counts(ctx)
    atoms = np.empty((np_, 2), np.int32)
    free = np.empty(np_, np.uint8)
    circ = np.empty((np_, 7), np.float64)
    verts = np.empty((nv, 3), np.float64)
    _check(load().eses_patch_data(ctx, _ptr(atoms), _ptr(free), _ptr(circ), _ptr(verts)), ctx)
    return {"pair_atoms": atoms, "pair_free": free, "pair_circle": circ, "vertices": verts}


def eses_crossing_edges_noalloc(labels, dims, idx0, idx1, idx2, capacity, stream=0):
    """Crossing edges of a device label grid into caller-allocated device
    outputs, with no allocation inside the library.  Returns the per-axis
    counts (numpy int64[3]); raises EsesError on failure."""
    d = np.ascontiguousarray(dims, dtype=np.int64)
    cap = np.ascontiguousarray(capacity, dtype=np.int64)
    counts = np.zeros(3, np.int64)
    rc = load().eses_crossing_edges_noalloc(_ptr(labels), _ptr(d), _ptr(idx0), _ptr(idx1), _ptr(idx2), _ptr(cap),
                                            _ptr(counts), ctypes.c_void_p(int(stream)) if stream else None)
    if rc != ESES_OK:
        raise EsesError(rc, f"eses_crossing_edges_noalloc failed (counts {counts.tolist()})")
    return counts


def eses_destroy(ctx):
    if ctx:
        load().eses_destroy(ctx)


class Surface:
    """Convenience wrapper: one molecule, one context."""

    def __init__(self, xyz, radii, r_p=1.4, h=0.5, margin=1.0, precision=ESES_PREC_FP32_FILTERED):
        self.ctx = eses_create(xyz, radii, r_p, h, margin)
        eses_set_option(self.ctx, ESES_OPT_PRECISION, precision)

    def run(self):
        eses_run(self.ctx)
        return self

    def grid(self):
        return eses_grid(self.ctx)

    def labels(self):
        return eses_labels(self.ctx)

    def intersections(self, axis):
        return eses_intersections(self.ctx, axis)

    def area_volume(self):
        return eses_area_volume(self.ctx)

    def stats(self):
        return eses_stats(self.ctx)

    def close(self):
        if self.ctx:
            eses_destroy(self.ctx)
            self.ctx = None

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
