"""Python binding of the C ABI in include/rll.h (ctypes; argument marshalling
only -- every step of the method runs in the CUDA library).

Arrays are passed as device pointers taken from contiguous torch CUDA tensors
(or as raw integer addresses / host numpy arrays where the C call says
"host"). The library is loaded from paper_1911_10217_gb300/_build/librll.so;
there is no fallback: if it is missing, import of this module's functions
raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

RLL_OK = 0
ERRORS = {1: "RLL_E_INVALID", 2: "RLL_E_NOMEM", 3: "RLL_E_CUDA", 4: "RLL_E_TABLE_FULL",
          8: "RLL_E_TIMEOUT", 16: "RLL_E_DEVICE"}
PREC = {"fp32": 0, "fp16": 1, "bf16": 2}
MODE = {"descent": 0, "uniform": 1, "descent2": 2}
REWARD = {"cluster": 0, "literal": 1}
BUILDER = {"lbvh": 0, "saoh": 1, "median": 2}

# every symbol declared in include/rll.h
EXPORTS = [
    "rll_ctx_create", "rll_ctx_set_stream", "rll_ctx_set_option", "rll_ctx_destroy", "rll_last_error", "rll_sync_status",
    "rll_build_light_tree", "rll_build_light_tree_ex", "rll_tree_update_emission", "rll_tree_num_lights", "rll_tree_export",
    "rll_tree_destroy", "rll_create_grid", "rll_grid_cut_len", "rll_grid_touched_cells", "rll_grid_export", "rll_grid_import",
    "rll_grid_destroy", "rll_sample_and_shade", "rll_sample_and_shade_ex", "rll_sample_and_shade_fp",
    "rll_sample_power", "rll_bounce_vertices",
    "rll_learn_update", "rll_learn_update_noalloc", "rll_learn_update_split", "rll_split_collapse",
    "rll_render_pass_host",
    "rll_batch_reserve", "rll_batch_set_items", "rll_batch_create", "rll_batch_set_config", "rll_batch_tune", "rll_batch_run", "rll_batch_capture",
    "rll_batch_launch", "rll_batch_destroy",
]


class RllError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class GridParams(ctypes.Structure):
    _fields_ = [("table_size", ctypes.c_uint32), ("cut_size", ctypes.c_uint32),
                ("origin", ctypes.c_float * 3), ("cell_size", ctypes.c_float),
                ("normal_bins", ctypes.c_uint32), ("jitter", ctypes.c_uint32),
                ("precision", ctypes.c_uint32), ("in_cluster_mode", ctypes.c_uint32),
                ("reward_mode", ctypes.c_uint32), ("alpha", ctypes.c_float),
                ("threshold", ctypes.c_float), ("eps", ctypes.c_float), ("q_init", ctypes.c_float),
                ("split_iterations", ctypes.c_uint32), ("levels", ctypes.c_uint32)]


class BatchItem(ctypes.Structure):
    _fields_ = [("grid", ctypes.c_void_p), ("tree", ctypes.c_void_p), ("pos", ctypes.c_void_p),
                ("nrm", ctypes.c_void_p), ("albedo", ctypes.c_void_p), ("n_points", ctypes.c_int64),
                ("boxes", ctypes.c_void_p), ("n_boxes", ctypes.c_int32), ("seed", ctypes.c_uint64),
                ("frame", ctypes.c_uint32), ("spp", ctypes.c_int32), ("rgb", ctypes.c_void_p)]


class SampleDebug(ctypes.Structure):
    _fields_ = [("light", ctypes.c_void_p), ("p_cut", ctypes.c_void_p), ("p_in", ctypes.c_void_p)]


_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load librll.so (building it first if asked and absent)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise RuntimeError(f"CUDA library not built: {path}")
        _build.build()
    L = ctypes.CDLL(path)
    P, I32, I64, U32, U64 = (ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_uint32,
                             ctypes.c_uint64)
    L.rll_ctx_create.argtypes = [ctypes.POINTER(P), ctypes.c_int, P]
    L.rll_ctx_set_stream.argtypes = [P, P]
    L.rll_ctx_set_option.argtypes = [P, ctypes.c_char_p, I64]
    L.rll_ctx_destroy.argtypes = [P]
    L.rll_last_error.argtypes = [P]
    L.rll_last_error.restype = ctypes.c_char_p
    L.rll_sync_status.argtypes = [P]
    L.rll_build_light_tree.argtypes = [P, P, P, I64, ctypes.POINTER(P)]
    L.rll_build_light_tree_ex.argtypes = [P, P, P, I64, I32, ctypes.POINTER(P)]
    L.rll_tree_update_emission.argtypes = [P, P, P]
    L.rll_tree_num_lights.argtypes = [P]
    L.rll_tree_num_lights.restype = I64
    L.rll_tree_export.argtypes = [P, P, P, P, P, P, P, P, P]
    L.rll_tree_destroy.argtypes = [P]
    L.rll_create_grid.argtypes = [P, P, ctypes.POINTER(GridParams), ctypes.POINTER(P)]
    L.rll_grid_cut_len.argtypes = [P]
    L.rll_grid_cut_len.restype = U32
    L.rll_grid_touched_cells.argtypes = [P, P, ctypes.POINTER(I64)]
    L.rll_grid_export.argtypes = [P, P, P, P, P, P]
    L.rll_grid_import.argtypes = [P, P, P, P, P, P]
    L.rll_grid_destroy.argtypes = [P]
    L.rll_sample_and_shade.argtypes = [P, P, P, P, P, P, I64, P, I32, U64, U32, I32, P, P, P]
    L.rll_sample_and_shade_ex.argtypes = [P, P, P, P, P, P, I64, P, I32, U64, U32, I32, P, P, P,
                                          ctypes.POINTER(SampleDebug)]
    L.rll_sample_and_shade_fp.argtypes = [P, P, P, P, P, P, P, I64, P, I32, U64, U32, I32, P, P, P, P]
    L.rll_sample_power.argtypes = [P, P, P, P, P, I64, P, I32, U64, U32, I32, P, P]
    L.rll_bounce_vertices.argtypes = [P, P, P, I64, P, I32, P, U64, U32, ctypes.c_float, P, P, P]
    L.rll_learn_update.argtypes = [P, P, P, P, I64]
    L.rll_learn_update_noalloc.argtypes = [P, P, P, P, I64]
    L.rll_learn_update_split.argtypes = [P, P, P, P, P, I64]
    L.rll_split_collapse.argtypes = [P, P, P]
    L.rll_render_pass_host.argtypes = [P, P, P, P, P, P, I64, P, I32, U64, U32, I32, I32, P]
    L.rll_batch_create.argtypes = [P, ctypes.POINTER(BatchItem), I32, ctypes.POINTER(P)]
    L.rll_batch_reserve.argtypes = [P, I32, I64, I64, ctypes.POINTER(P)]
    L.rll_batch_set_items.argtypes = [P, P, ctypes.POINTER(BatchItem), I32]
    L.rll_batch_set_config.argtypes = [P, P, I32, I32]
    L.rll_batch_tune.argtypes = [P, P, ctypes.POINTER(I32), ctypes.POINTER(I32)]
    L.rll_batch_run.argtypes = [P, P, I32]
    L.rll_batch_capture.argtypes = [P, P, I32]
    L.rll_batch_launch.argtypes = [P, P]
    L.rll_batch_destroy.argtypes = [P]
    _lib = L
    return L


def _ptr(x):
    """Device (or host) address of a tensor / array / int / None."""
    if x is None:
        return None
    if isinstance(x, int):
        return x
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr()
    raise TypeError(f"cannot pass {type(x)} as a pointer")


def _check_tensor(t, dtype_name, device=True):
    if t is None:
        return
    if hasattr(t, "dtype"):
        if str(t.dtype).split(".")[-1] != dtype_name:
            raise TypeError(f"expected {dtype_name}, got {t.dtype}")
        if device and hasattr(t, "is_cuda") and not t.is_cuda:
            raise ValueError("expected a CUDA tensor")


class Context:
    """rll_ctx: a device and the CUDA stream work is enqueued on."""

    def __init__(self, device: int = 0, stream=None):
        self.lib = load()
        h = ctypes.c_void_p()
        rc = self.lib.rll_ctx_create(ctypes.byref(h), int(device), self._stream_ptr(stream))
        if rc != RLL_OK:
            raise RllError(rc, "rll_ctx_create failed")
        self.h = h
        self.device = device

    @staticmethod
    def _stream_ptr(stream):
        if stream is None:
            return None
        if isinstance(stream, int):
            return stream
        return stream.cuda_stream

    def set_stream(self, stream):
        self._check(self.lib.rll_ctx_set_stream(self.h, self._stream_ptr(stream)))

    def set_option(self, name: str, value: int):
        self._check(self.lib.rll_ctx_set_option(self.h, name.encode(), int(value)))

    def _check(self, rc):
        if rc != RLL_OK:
            raise RllError(rc, self.lib.rll_last_error(self.h).decode())

    def sync_status(self) -> int:
        r = self.lib.rll_sync_status(self.h)
        if r < 0:
            raise RllError(-r, self.lib.rll_last_error(self.h).decode())
        return r

    def close(self):
        if getattr(self, "h", None):
            self.lib.rll_ctx_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Tree:
    """rll_tree built by rll_build_light_tree_ex (builder "lbvh", "saoh" or "median")."""

    def __init__(self, ctx: Context, tri, emission, builder: str = "lbvh"):
        _check_tensor(tri, "float32")
        _check_tensor(emission, "float32")
        n = int(tri.shape[0])
        h = ctypes.c_void_p()
        ctx._check(ctx.lib.rll_build_light_tree_ex(ctx.h, _ptr(tri), _ptr(emission), n, BUILDER[builder],
                                                   ctypes.byref(h)))
        self.ctx, self.h, self.n, self.builder = ctx, h, n, builder

    def update_emission(self, emission):
        _check_tensor(emission, "float32")
        self.ctx._check(self.ctx.lib.rll_tree_update_emission(self.ctx.h, self.h, _ptr(emission)))

    def export(self):
        n = self.n
        nn = 2 * n - 1
        out = dict(perm=np.zeros(n, np.uint32), left=np.zeros(max(n - 1, 1), np.int32),
                   right=np.zeros(max(n - 1, 1), np.int32), parent=np.zeros(nn, np.int32),
                   begin=np.zeros(nn, np.uint32), end=np.zeros(nn, np.uint32),
                   rec=np.zeros((nn, 11), np.float32))
        self.ctx._check(self.ctx.lib.rll_tree_export(
            self.ctx.h, self.h, *[_ptr(out[k]) for k in ("perm", "left", "right", "parent", "begin",
                                                         "end", "rec")]))
        return out

    def close(self):
        if getattr(self, "h", None):
            self.ctx.lib.rll_tree_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def grid_params(table_size, cut_size, origin=(0.0, 0.0, 0.0), cell_size=1.0, normal_bins=1,
                jitter=False, precision="fp32", mode="descent", reward="cluster", alpha=0.03,
                threshold=2.0, eps=0.02, q_init=1e-3, split_iterations=1, levels=1) -> GridParams:
    return GridParams(int(table_size), int(cut_size), (ctypes.c_float * 3)(*origin), float(cell_size),
                      int(normal_bins), int(bool(jitter)), PREC[precision], MODE[mode], REWARD[reward],
                      float(alpha), float(threshold), float(eps), float(q_init), int(split_iterations),
                      int(levels))


def grid_params_for(grid_config, **overrides) -> GridParams:
    """GridParams of a scene's grid configuration (scenes.GridConfig)."""
    g = grid_config
    args = dict(table_size=g.table_size, cut_size=g.cut_size, origin=g.origin, cell_size=g.cell_size,
                normal_bins=g.normal_bins, jitter=g.jitter, q_init=g.q_init, alpha=g.alpha, eps=g.eps,
                threshold=g.threshold, split_iterations=g.split_iterations, levels=g.levels)
    args.update(overrides)
    return grid_params(**args)


class Grid:
    """rll_grid created by rll_create_grid."""

    def __init__(self, ctx: Context, tree: Tree, params: GridParams):
        h = ctypes.c_void_p()
        ctx._check(ctx.lib.rll_create_grid(ctx.h, tree.h, ctypes.byref(params), ctypes.byref(h)))
        self.ctx, self.h, self.tree, self.params = ctx, h, tree, params
        self.levels = max(1, int(params.levels))
        self.H, self.M = int(params.table_size) * self.levels, int(params.cut_size)
        self.m = int(ctx.lib.rll_grid_cut_len(h))

    def touched_cells(self) -> int:
        """Cells rewritten by the last learning call (synchronises)."""
        n = ctypes.c_int64()
        self.ctx._check(self.ctx.lib.rll_grid_touched_cells(self.ctx.h, self.h, ctypes.byref(n)))
        return int(n.value)

    def export(self):
        H, M = self.H, self.M
        out = dict(keys=np.zeros(H, np.uint64), cut=np.zeros((H, M), np.int32),
                   q=np.zeros((H, M), np.float32), c=np.zeros((H, M), np.float32))
        self.ctx._check(self.ctx.lib.rll_grid_export(self.ctx.h, self.h, _ptr(out["keys"]),
                                                     _ptr(out["cut"]), _ptr(out["q"]),
                                                     _ptr(out["c"])))
        return out

    def import_state(self, keys, cut, q, c):
        keys = np.ascontiguousarray(keys, np.uint64)
        cut = np.ascontiguousarray(cut, np.int32)
        q = np.ascontiguousarray(q, np.float32)
        c = np.ascontiguousarray(c, np.float32)
        self.ctx._check(self.ctx.lib.rll_grid_import(self.ctx.h, self.h, _ptr(keys), _ptr(cut),
                                                     _ptr(q), _ptr(c)))

    def close(self):
        if getattr(self, "h", None):
            self.ctx.lib.rll_grid_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def sample_and_shade(ctx: Context, grid: Grid, tree: Tree, pos, nrm, albedo, boxes, seed, frame, spp,
                     rgb, rec_key=None, rec_val=None, dbg_light=None, dbg_pcut=None, dbg_pin=None,
                     footprint=None):
    for t, d in ((pos, "float32"), (nrm, "float32"), (albedo, "float32"), (boxes, "float32"),
                 (rgb, "float32"), (rec_key, "int32"), (rec_val, "float32"), (footprint, "float32")):
        _check_tensor(t, d)
    n = int(albedo.shape[0])
    k = int(boxes.shape[0]) if boxes is not None else 0
    if footprint is not None:
        dbg = SampleDebug(_ptr(dbg_light), _ptr(dbg_pcut), _ptr(dbg_pin))
        ctx._check(ctx.lib.rll_sample_and_shade_fp(ctx.h, grid.h, tree.h, _ptr(pos), _ptr(nrm),
                                                   _ptr(albedo), _ptr(footprint), n, _ptr(boxes), k,
                                                   int(seed), int(frame), int(spp), _ptr(rgb),
                                                   _ptr(rec_key), _ptr(rec_val), ctypes.byref(dbg)))
    elif dbg_light is None and dbg_pcut is None and dbg_pin is None:
        ctx._check(ctx.lib.rll_sample_and_shade(ctx.h, grid.h, tree.h, _ptr(pos), _ptr(nrm),
                                                _ptr(albedo), n, _ptr(boxes), k, int(seed),
                                                int(frame), int(spp), _ptr(rgb), _ptr(rec_key),
                                                _ptr(rec_val)))
    else:
        dbg = SampleDebug(_ptr(dbg_light), _ptr(dbg_pcut), _ptr(dbg_pin))
        ctx._check(ctx.lib.rll_sample_and_shade_ex(ctx.h, grid.h, tree.h, _ptr(pos), _ptr(nrm),
                                                   _ptr(albedo), n, _ptr(boxes), k, int(seed),
                                                   int(frame), int(spp), _ptr(rgb), _ptr(rec_key),
                                                   _ptr(rec_val), ctypes.byref(dbg)))


def sample_power(ctx: Context, tree: Tree, pos, nrm, albedo, boxes, seed, frame, spp, rgb,
                 light_out=None):
    n = int(albedo.shape[0])
    k = int(boxes.shape[0]) if boxes is not None else 0
    ctx._check(ctx.lib.rll_sample_power(ctx.h, tree.h, _ptr(pos), _ptr(nrm), _ptr(albedo), n,
                                        _ptr(boxes), k, int(seed), int(frame), int(spp), _ptr(rgb),
                                        _ptr(light_out)))


def bounce_vertices(ctx: Context, pos, nrm, boxes, room, seed, frame, paths_per_tile, out_pos, out_nrm,
                    out_footprint):
    """rll_bounce_vertices: one diffuse bounce from every point; room is a
    host sequence of 6 floats (min xyz, max xyz)."""
    P = int(pos.shape[1])
    for t in (pos, nrm, out_pos, out_nrm):
        _check_tensor(t, "float32")
    _check_tensor(out_footprint, "float32")
    rm = np.ascontiguousarray(np.asarray(room, np.float32).reshape(6))
    ctx._check(ctx.lib.rll_bounce_vertices(ctx.h, _ptr(pos), _ptr(nrm), P, _ptr(boxes), int(boxes.shape[0]),
                                           _ptr(rm), int(seed), int(frame), float(paths_per_tile),
                                           _ptr(out_pos), _ptr(out_nrm), _ptr(out_footprint)))


def learn_update(ctx: Context, grid: Grid, rec_key, rec_val, n_records=None):
    n = int(rec_key.shape[0]) if n_records is None else int(n_records)
    ctx._check(ctx.lib.rll_learn_update(ctx.h, grid.h, _ptr(rec_key), _ptr(rec_val), n))


def learn_update_split(ctx: Context, grid: Grid, tree: Tree, rec_key, rec_val, n_records=None):
    """rll_learn_update_split: learn_update then split_collapse, fused per cell."""
    n = int(rec_key.shape[0]) if n_records is None else int(n_records)
    ctx._check(ctx.lib.rll_learn_update_split(ctx.h, grid.h, tree.h, _ptr(rec_key), _ptr(rec_val), n))


def split_collapse(ctx: Context, grid: Grid, tree: Tree):
    ctx._check(ctx.lib.rll_split_collapse(ctx.h, grid.h, tree.h))


def render_pass_host(ctx: Context, grid: Grid, tree: Tree, pos, nrm, albedo, boxes, seed, frame,
                     spp, rgb, do_split=True):
    """Whole pass from HOST buffers (numpy or pinned CPU tensors)."""
    n = int(albedo.shape[0])
    k = int(boxes.shape[0])
    ctx._check(ctx.lib.rll_render_pass_host(ctx.h, grid.h, tree.h, _ptr(pos), _ptr(nrm),
                                            _ptr(albedo), n, _ptr(boxes), k, int(seed), int(frame),
                                            int(spp), int(bool(do_split)), _ptr(rgb)))


class Batch:
    """rll_batch: many scenes sampled by one persistent launch per stage.
    `items` is a list of dicts with keys grid, tree, pos, nrm, albedo, boxes,
    seed, frame, spp, rgb (device tensors for the arrays)."""

    def __init__(self, ctx: Context, items=None, max_items=None, max_records=None, max_cells=None):
        h = ctypes.c_void_p()
        if items is not None:
            ctx._check(ctx.lib.rll_batch_create(ctx.h, self._array(items), len(items), ctypes.byref(h)))
        else:
            ctx._check(ctx.lib.rll_batch_reserve(ctx.h, int(max_items), int(max_records), int(max_cells),
                                                 ctypes.byref(h)))
        self.ctx, self.h, self.items = ctx, h, items

    @staticmethod
    def _array(items):
        arr = (BatchItem * len(items))()
        for i, it in enumerate(items):
            arr[i] = BatchItem(it["grid"].h.value, it["tree"].h.value, _ptr(it["pos"]), _ptr(it["nrm"]),
                               _ptr(it["albedo"]), int(it["albedo"].shape[0]), _ptr(it["boxes"]),
                               int(it["boxes"].shape[0]), int(it["seed"]), int(it.get("frame", 0)),
                               int(it.get("spp", 1)), _ptr(it["rgb"]))
        return arr

    def set_items(self, items):
        self.ctx._check(self.ctx.lib.rll_batch_set_items(self.ctx.h, self.h, self._array(items), len(items)))
        self.items = items

    def set_config(self, tile_points, min_blocks):
        self.ctx._check(self.ctx.lib.rll_batch_set_config(self.ctx.h, self.h, int(tile_points), int(min_blocks)))

    def tune(self):
        tp, mb = ctypes.c_int32(), ctypes.c_int32()
        self.ctx._check(self.ctx.lib.rll_batch_tune(self.ctx.h, self.h, ctypes.byref(tp), ctypes.byref(mb)))
        return tp.value, mb.value

    def run(self, do_split=True):
        self.ctx._check(self.ctx.lib.rll_batch_run(self.ctx.h, self.h, int(bool(do_split))))

    def capture(self, do_split=True):
        self.ctx._check(self.ctx.lib.rll_batch_capture(self.ctx.h, self.h, int(bool(do_split))))

    def launch(self):
        self.ctx._check(self.ctx.lib.rll_batch_launch(self.ctx.h, self.h))

    def close(self):
        if getattr(self, "h", None):
            self.ctx.lib.rll_batch_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
