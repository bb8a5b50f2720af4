"""ctypes wrapper of the CPU oracle (rll_oracle.c).

Test infrastructure only: the tests, the smoke check and the benchmark's
CPU-baseline leg are the only callers. Arrays are numpy; the compiled library
lives in oracle/_build/ and is built on first use (or by build()).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rll_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)
PREC = {"fp32": 0, "fp16": 1, "bf16": 2}
MODE = {"descent": 0, "uniform": 1, "descent2": 2}
REWARD = {"cluster": 0, "literal": 1}
BUILDER = {"lbvh": 0, "saoh": 1, "median": 2}


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no fused multiply-add)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


class _Tree(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("perm", ctypes.c_void_p), ("code", ctypes.c_void_p),
                ("left", ctypes.c_void_p), ("right", ctypes.c_void_p), ("parent", ctypes.c_void_p),
                ("begin", ctypes.c_void_p), ("end", ctypes.c_void_p), ("rec", ctypes.c_void_p),
                ("phi64", ctypes.c_void_p)]


class _Grid(ctypes.Structure):
    _fields_ = [("H", ctypes.c_uint32), ("M", ctypes.c_uint32), ("m", ctypes.c_uint32),
                ("origin", ctypes.c_float * 3), ("h", ctypes.c_float), ("nb", ctypes.c_uint32),
                ("jitter", ctypes.c_uint32), ("mode", ctypes.c_uint32),
                ("reward_mode", ctypes.c_uint32), ("precision", ctypes.c_uint32),
                ("alpha", ctypes.c_double), ("T", ctypes.c_double), ("eps", ctypes.c_double),
                ("keys", ctypes.c_void_p), ("cut", ctypes.c_void_p), ("Q", ctypes.c_void_p),
                ("C", ctypes.c_void_p), ("def_cut", ctypes.c_void_p), ("def_Q", ctypes.c_void_p),
                ("def_C", ctypes.c_void_p), ("levels", ctypes.c_uint32), ("Hl", ctypes.c_uint32)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = ctypes.CDLL(build())
            P = ctypes.c_void_p
            L.orc_philox4x32_10.argtypes = [P, P, P]
            L.orc_build_tree.argtypes = [ctypes.c_int64, P, P, ctypes.POINTER(_Tree)]
            L.orc_build_tree_ex.argtypes = [ctypes.c_int64, P, P, ctypes.POINTER(_Tree), ctypes.c_int]
            L.orc_initial_cut.argtypes = [ctypes.POINTER(_Tree), ctypes.c_int, P]
            L.orc_initial_cut.restype = ctypes.c_int
            L.orc_cdf.argtypes = [ctypes.c_int, P, ctypes.c_double, ctypes.c_int, P]
            L.orc_round_storage.argtypes = [ctypes.c_double, ctypes.c_int]
            L.orc_round_storage.restype = ctypes.c_double
            L.orc_cell_key.argtypes = [ctypes.POINTER(_Grid), P, P, P]
            L.orc_cell_key.restype = ctypes.c_uint64
            L.orc_fmix64.argtypes = [ctypes.c_uint64]
            L.orc_fmix64.restype = ctypes.c_uint64
            L.orc_lookup_insert.argtypes = [ctypes.POINTER(_Grid), ctypes.c_uint64]
            L.orc_lookup_insert.restype = ctypes.c_int64
            L.orc_importance32.argtypes = [P, P, P, P, P]
            L.orc_bounce_vertices.argtypes = [ctypes.c_int64, P, P, ctypes.c_int, P, P, ctypes.c_uint64,
                                              ctypes.c_uint32, ctypes.c_float, P, P, P]
            L.orc_node_consts32.argtypes = [P, P]
            L.orc_bound64.argtypes = [P, ctypes.c_double, ctypes.c_double, ctypes.c_double, P,
                                      ctypes.c_double, P, P]
            L.orc_bound64.restype = ctypes.c_double
            L.orc_half_round.argtypes = [ctypes.c_float, ctypes.c_int]
            L.orc_shadow32.argtypes = [P, P, ctypes.c_int, P]
            L.orc_shadow64.argtypes = [P, P, ctypes.c_int, P]
            L.orc_half_round.restype = ctypes.c_float
            L.orc_sample_frame.argtypes = [ctypes.POINTER(_Tree), P, P, ctypes.c_int, P,
                                           ctypes.POINTER(_Grid), ctypes.c_int64, P, P, P, P,
                                           ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int,
                                           P, P, P, P, P, P, P, P, P, ctypes.c_int64, ctypes.c_int64]
            L.orc_footprint_level.argtypes = [ctypes.c_float, ctypes.c_float, ctypes.c_uint32]
            L.orc_footprint_level.restype = ctypes.c_uint32
            L.orc_cell_key_level.argtypes = [ctypes.POINTER(_Grid), ctypes.c_uint32, P, P, P]
            L.orc_cell_key_level.restype = ctypes.c_uint64
            L.orc_learn.argtypes = [ctypes.POINTER(_Grid), ctypes.c_int64, P, P, P, P]
            L.orc_split_collapse_cell.argtypes = [ctypes.POINTER(_Tree), ctypes.c_int, P, P,
                                                  ctypes.c_double, ctypes.c_double, ctypes.c_int,
                                                  ctypes.c_int, P]
            L.orc_split_collapse_cell.restype = ctypes.c_int
            L.orc_light_pdf.argtypes = [ctypes.POINTER(_Tree), ctypes.c_int, ctypes.c_int, P, P,
                                        P, P, ctypes.c_int64]
            L.orc_light_pdf.restype = ctypes.c_double
            L.orc_sample_power.argtypes = [ctypes.POINTER(_Tree), P, P, ctypes.c_int, P,
                                           ctypes.c_int64, P, P, P, ctypes.c_uint64,
                                           ctypes.c_uint32, ctypes.c_int, P, P, ctypes.c_int64,
                                           ctypes.c_int64]
            L.orc_direct_bruteforce.argtypes = [P, P, ctypes.c_float, ctypes.c_int64, P, P,
                                                ctypes.c_int, P, ctypes.c_int, P]
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _f32(a):
    return np.ascontiguousarray(a, dtype=np.float32)


def philox4x32_10(counter, key):
    c = np.asarray(counter, np.uint32).copy()
    k = np.asarray(key, np.uint32).copy()
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def round_storage(v, precision="fp32"):
    return lib().orc_round_storage(float(v), PREC[precision])


class Tree:
    """The oracle's light tree (node numbering: internal 0..n-2, leaf of
    sorted light l is n-1+l, root 0)."""

    def __init__(self, tris, emission, builder="lbvh"):
        tris = _f32(tris).reshape(-1, 9)
        emission = _f32(emission).reshape(-1, 3)
        n = tris.shape[0]
        nn = 2 * n - 1
        self.n = n
        self.tris = tris
        self.emission = emission
        self.perm = np.zeros(n, np.uint32)
        self.code = np.zeros(n, np.uint32)
        self.left = np.full(max(n - 1, 1), -1, np.int32)
        self.right = np.full(max(n - 1, 1), -1, np.int32)
        self.parent = np.full(nn, -1, np.int32)
        self.begin = np.zeros(nn, np.uint32)
        self.end = np.zeros(nn, np.uint32)
        self.rec = np.zeros((nn, 11), np.float32)
        self.phi64 = np.zeros(nn, np.float64)
        self._s = _Tree(n, _p(self.perm), _p(self.code), _p(self.left), _p(self.right),
                        _p(self.parent), _p(self.begin), _p(self.end), _p(self.rec),
                        _p(self.phi64))
        self.builder = builder
        rc = lib().orc_build_tree_ex(n, _p(tris), _p(emission), ctypes.byref(self._s), BUILDER[builder])
        if rc != 0:
            raise RuntimeError("oracle tree build failed")

    def initial_cut(self, M):
        cut = np.zeros(max(M, 1), np.int32)
        m = lib().orc_initial_cut(ctypes.byref(self._s), int(M), _p(cut))
        return cut[:m].copy()

    def is_leaf(self, node):
        return node >= self.n - 1

    def importance(self, node, x, nrm):
        """The descent bound of a node at (x, nrm): num / den (binary32 parts)."""
        num, den = ctypes.c_float(), ctypes.c_float()
        lib().orc_importance32(_p(np.ascontiguousarray(self.rec[node])), _p(_f32(x)), _p(_f32(nrm)),
                               ctypes.byref(num), ctypes.byref(den))
        return float(num.value) / float(den.value)


def bounce_vertices(pos, nrm, boxes, room, seed, frame, paths_per_tile):
    """One diffuse bounce per point (cosine-weighted direction, nearest box
    face or room wall): vertex positions and face normals SoA [3][P] and
    footprints [P] (binary32)."""
    pos, nrm = _f32(pos), _f32(nrm)
    P = pos.shape[1]
    boxes = _f32(boxes).reshape(-1, 6)
    y, ny, fp = np.zeros((3, P), np.float32), np.zeros((3, P), np.float32), np.zeros(P, np.float32)
    lib().orc_bounce_vertices(P, _p(pos), _p(nrm), int(boxes.shape[0]), _p(boxes), _p(_f32(room)),
                              int(seed), int(frame), float(paths_per_tile), _p(y), _p(ny), _p(fp))
    return y, ny, fp


def node_consts(rec):
    """Compact bound constants of a node record: centre xyz, r, r*r, cone
    cos and sin (binary32 values)."""
    k = np.zeros(7, np.float32)
    lib().orc_node_consts32(_p(_f32(rec)), _p(k))
    return k


def bound64(centre, r, cos_t, sin_t, axis, phi, x, nrm):
    """The descent bound written out plainly in double precision."""
    c = np.ascontiguousarray(centre, np.float64)
    a = np.ascontiguousarray(axis, np.float64)
    xx = np.ascontiguousarray(x, np.float64)
    nn = np.ascontiguousarray(nrm, np.float64)
    return float(lib().orc_bound64(_p(c), float(r), float(cos_t), float(sin_t), _p(a), float(phi), _p(xx), _p(nn)))


def occluded32(o, y, boxes):
    """The binary32 shadow test of the sampler: segment o -> y (t in (0,
    0.9999)) against boxes [K][6]."""
    o = np.ascontiguousarray(o, np.float32)
    y = np.ascontiguousarray(y, np.float32)
    b = np.ascontiguousarray(boxes, np.float32).reshape(-1, 6)
    return bool(lib().orc_shadow32(_p(o), _p(y), int(b.shape[0]), _p(b)))


def occluded64(o, y, boxes):
    """The double shadow test of the brute-force reference (same segment)."""
    o = np.ascontiguousarray(o, np.float64)
    y = np.ascontiguousarray(y, np.float64)
    b = np.ascontiguousarray(boxes, np.float32).reshape(-1, 6)
    return bool(lib().orc_shadow64(_p(o), _p(y), int(b.shape[0]), _p(b)))


def half_round(x, up):
    """x rounded to binary16 toward +inf (up) or -inf, as a float."""
    return float(lib().orc_half_round(float(x), 1 if up else 0))


def footprint_level(footprint, cell_size, levels):
    """Resolution level of a point with this footprint (binary32)."""
    return int(lib().orc_footprint_level(float(np.float32(footprint)), float(np.float32(cell_size)),
                                         int(levels)))


def cdf(q, eps=0.01, precision="fp32"):
    q = np.ascontiguousarray(q, np.float64)
    out = np.zeros_like(q)
    lib().orc_cdf(len(q), _p(q), float(eps), PREC[precision], _p(out))
    return out


class Grid:
    """The oracle's hash grid: H slots of (key, cut[M], Q[M], C[M]); Q and C
    hold table-precision values in double. With levels > 1 the grid is
    multi-resolution: levels tables of table_size slots (H = levels *
    table_size), level l of cell size cell_size * 2^l, chosen per point from
    its footprint (sample_frame's footprint argument)."""

    def __init__(self, tree: Tree, table_size, cut_size, origin=(0, 0, 0), cell_size=1.0,
                 normal_bins=1, jitter=False, mode="descent", reward="cluster", precision="fp32",
                 alpha=0.03, T=2.0, eps=0.02, q_init=1e-3, split_iterations=1, levels=1):
        self.tree = tree
        Hl, M = int(table_size), int(cut_size)
        assert Hl & (Hl - 1) == 0
        levels = max(1, int(levels))
        H = Hl * levels
        self.def_cut = tree.initial_cut(M)
        m = len(self.def_cut)
        self.def_Q = np.array([round_storage(q_init, precision)] * m, np.float64)
        self.def_C = cdf(self.def_Q, eps, precision)
        self.keys = np.full(H, EMPTY, np.uint64)
        self.cut = np.zeros((H, M), np.int32)
        self.Q = np.zeros((H, M), np.float64)
        self.C = np.zeros((H, M), np.float64)
        self.H, self.M, self.m = H, M, m
        self.precision = precision
        self.params = dict(origin=tuple(float(o) for o in origin), cell_size=float(cell_size),
                           normal_bins=int(normal_bins), jitter=bool(jitter), mode=mode,
                           reward=reward, precision=precision, alpha=float(alpha), T=float(T),
                           eps=float(eps), q_init=float(q_init),
                           split_iterations=int(split_iterations), levels=levels)
        self.levels, self.Hl = levels, Hl
        self._s = _Grid(H, M, m, (ctypes.c_float * 3)(*origin), float(cell_size), int(normal_bins),
                        int(bool(jitter)), MODE[mode], REWARD[reward], PREC[precision],
                        float(alpha), float(T), float(eps), _p(self.keys), _p(self.cut),
                        _p(self.Q), _p(self.C), _p(self.def_cut), _p(self.def_Q), _p(self.def_C),
                        levels, Hl)

    @classmethod
    def for_scene(cls, tree, scene, **kw):
        g = scene.grid
        args = dict(table_size=g.table_size, cut_size=g.cut_size, origin=g.origin,
                    cell_size=g.cell_size, normal_bins=g.normal_bins, jitter=g.jitter,
                    q_init=g.q_init, alpha=g.alpha, eps=g.eps, T=g.threshold,
                    split_iterations=g.split_iterations, levels=g.levels)
        args.update(kw)
        return cls(tree, **args)

    def copy_state_from(self, keys, cut, Q, C):
        self.keys[...] = keys
        self.cut[...] = cut
        self.Q[...] = Q
        self.C[...] = C

    def cell_key(self, x, nrm, jit=(0, 0, 0, 0, 0)):
        return lib().orc_cell_key(ctypes.byref(self._s), _p(_f32(x)), _p(_f32(nrm)),
                                  _p(_f32(jit)))

    def cell_key_level(self, level, x, nrm, jit=(0, 0, 0, 0, 0)):
        return lib().orc_cell_key_level(ctypes.byref(self._s), int(level), _p(_f32(x)), _p(_f32(nrm)),
                                        _p(_f32(jit)))

    def lookup_insert(self, key):
        return lib().orc_lookup_insert(ctypes.byref(self._s), int(key))

    def sample_frame(self, scene_arrays, seed, frame, spp, first=0, count=-1, emission=None,
                     footprint=None):
        tris, emis, boxes, pos, nrm, albedo = scene_arrays
        if emission is not None:
            emis = emission
        npts = pos.shape[1]
        cnt = npts - first if count < 0 else count
        ns = cnt * spp
        out = dict(rgb=np.zeros((3, cnt)), light=np.zeros(ns, np.int64),
                   slot=np.zeros(ns, np.int64), s=np.zeros(ns, np.int32),
                   reward=np.zeros(ns), p_cut=np.zeros(ns), p_in=np.zeros(ns),
                   margin=np.zeros(ns), visible=np.zeros(ns, np.int32))
        lib().orc_sample_frame(ctypes.byref(self.tree._s), _p(_f32(tris)), _p(_f32(emis)),
                               int(boxes.shape[0]), _p(_f32(boxes)), ctypes.byref(self._s),
                               npts, _p(_f32(pos)), _p(_f32(nrm)), _p(_f32(albedo)),
                               None if footprint is None else _p(_f32(footprint)),
                               int(seed), int(frame), int(spp), _p(out["rgb"]),
                               _p(out["light"]), _p(out["slot"]), _p(out["s"]),
                               _p(out["reward"]), _p(out["p_cut"]), _p(out["p_in"]),
                               _p(out["margin"]), _p(out["visible"]), int(first), int(cnt))
        return out

    def learn(self, slot, s, reward):
        slot = np.ascontiguousarray(slot, np.int64)
        s = np.ascontiguousarray(s, np.int32)
        reward = np.ascontiguousarray(reward, np.float64)
        touched = np.zeros(self.H, np.uint8)
        lib().orc_learn(ctypes.byref(self._s), len(slot), _p(slot), _p(s), _p(reward), _p(touched))
        return touched.astype(bool)

    def split_collapse(self, touched):
        """Split-collapse every touched cell (up to split_iterations steps
        each); returns the number of cells changed."""
        changed = 0
        c_out = np.zeros(self.m)
        for slot in np.nonzero(touched)[0]:
            cut = np.ascontiguousarray(self.cut[slot, :self.m])
            q = np.ascontiguousarray(self.Q[slot, :self.m])
            steps = lib().orc_split_collapse_cell(ctypes.byref(self.tree._s), self.m, _p(cut), _p(q),
                                                  self.params["T"], self.params["eps"],
                                                  PREC[self.precision], self.params["split_iterations"],
                                                  _p(c_out))
            changed += steps > 0
            self.cut[slot, :self.m] = cut
            self.Q[slot, :self.m] = q
            self.C[slot, :self.m] = c_out
        return changed

    def light_pdf(self, slot, x, nrm, light):
        cut = np.ascontiguousarray(self.cut[slot, :self.m]) if slot >= 0 else self.def_cut
        C = np.ascontiguousarray(self.C[slot, :self.m]) if slot >= 0 else self.def_C
        return lib().orc_light_pdf(ctypes.byref(self.tree._s), MODE[self.params["mode"]], self.m,
                                   _p(np.ascontiguousarray(cut, np.int32)), _p(C), _p(_f32(x)),
                                   _p(_f32(nrm)), int(light))


def split_collapse_cell(tree: Tree, cut, q, T=2.0, eps=0.01, precision="fp32", max_iter=1):
    """Split-collapse of one cut row, at most max_iter steps; returns the new
    cut, Q, C and the number of steps that changed the cut."""
    cut = np.ascontiguousarray(cut, np.int32).copy()
    q = np.ascontiguousarray(q, np.float64).copy()
    c = np.zeros(len(cut))
    steps = lib().orc_split_collapse_cell(ctypes.byref(tree._s), len(cut), _p(cut), _p(q),
                                          float(T), float(eps), PREC[precision], int(max_iter), _p(c))
    return cut, q, c, int(steps)


def sample_power(tree: Tree, scene_arrays, seed, frame, spp, first=0, count=-1, emission=None):
    tris, emis, boxes, pos, nrm, albedo = scene_arrays
    if emission is not None:
        emis = emission
    npts = pos.shape[1]
    cnt = npts - first if count < 0 else count
    rgb = np.zeros((3, cnt))
    light = np.zeros(cnt * spp, np.int64)
    lib().orc_sample_power(ctypes.byref(tree._s), _p(_f32(tris)), _p(_f32(emis)),
                           int(boxes.shape[0]), _p(_f32(boxes)), npts, _p(_f32(pos)),
                           _p(_f32(nrm)), _p(_f32(albedo)), int(seed), int(frame), int(spp),
                           _p(rgb), _p(light), int(first), int(cnt))
    return rgb, light


def direct_bruteforce(x, nrm, albedo, tris, emission, boxes, level=5):
    out = np.zeros(3)
    boxes = _f32(boxes).reshape(-1, 6)
    lib().orc_direct_bruteforce(_p(_f32(x)), _p(_f32(nrm)), float(albedo),
                                int(_f32(tris).reshape(-1, 9).shape[0]),
                                _p(_f32(tris).reshape(-1, 9)), _p(_f32(emission).reshape(-1, 3)),
                                int(boxes.shape[0]), _p(boxes), int(level), _p(out))
    return out


def scene_arrays(scene, emission=None):
    """(tris, emission, boxes, pos, nrm, albedo) as contiguous float32."""
    return (_f32(scene.tris).reshape(-1, 9), _f32(scene.emission if emission is None else emission),
            _f32(scene.boxes).reshape(-1, 6), _f32(scene.pos), _f32(scene.nrm), _f32(scene.albedo))
