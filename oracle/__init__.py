"""FP64 CPU oracle for the straightest-geodesic exponential map (test infrastructure).

Only the test suite, ``__graft_entry__.smoke()`` and the benchmark's ``cpu_baseline`` /
``--impl reference`` legs may import this package.  The library under
``paper_2603_15780_gb300`` never imports it, and this package imports nothing from
the library: the two share only the seeded input generators in ``meshgen``.

The arithmetic lives in ``sgeo_oracle.c`` (plain C99, FP64, OpenMP over queries),
compiled on first use with gcc into ``oracle/_build/liboracle.so``.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sgeo_oracle.c")
_OUT = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None

# per-query status bits (same meaning as the library's status word)
BOUNDARY, MAX_STEPS, NEAR_VERTEX, NEAR_EDGE, VERTEX_HIT = 1, 2, 4, 8, 16
START_ON_EDGE, INVALID = 64, 128
HOLE = 2048          # hole avoidance traced along the boundary (boundary_mode=1)


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O3, no fp contraction so x86 and Arm agree)."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O3", "-std=c99", "-fopenmp", "-ffp-contract=off", "-shared",
                               "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


class _Opts(C.Structure):
    _fields_ = [("max_steps", C.c_int32), ("path_cap", C.c_int32), ("tau_snap", C.c_double),
                ("tau_near", C.c_double), ("boundary_mode", C.c_int32)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            P = C.c_void_p
            L.om_mesh_build.argtypes = [P, C.c_int64, P, C.c_int64, C.POINTER(P)]
            L.om_mesh_build.restype = C.c_int
            L.om_mesh_free.argtypes = [P]
            L.om_mesh_lref.argtypes = [P]
            L.om_mesh_lref.restype = C.c_double
            L.om_mesh_theta.argtypes = [P, P, P]
            L.om_mesh_adjacency.argtypes = [P, P]
            L.om_exp_map.argtypes = [P, C.c_int64, P, P, P, P, C.c_int32, P, P, P, P, P, P, P, P, P,
                                     P, P, P, P, P, C.POINTER(_Opts), C.c_int]
            L.om_ep_backward.argtypes = [P, C.c_int64, P, P, P, P, P, P, C.POINTER(_Opts), C.c_int]
            L.om_gfd_backward.argtypes = [P, C.c_int64, P, P, P, C.c_double, C.c_double, P, P, P, P,
                                          P, C.POINTER(_Opts), C.c_int]
            _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


class OracleError(RuntimeError):
    pass


class Mesh:
    """Oracle mesh: FP64 copy of (X, F) with adjacency, vertex angle sums and l_ref."""

    def __init__(self, X, F):
        self.X = _f64(X, (-1, 3))
        self.F = np.ascontiguousarray(F, dtype=np.int32).reshape(-1, 3)
        h = C.c_void_p()
        rc = lib().om_mesh_build(_p(self.X), len(self.X), _p(self.F), len(self.F), C.byref(h))
        if rc != 0:
            raise OracleError({1: "invalid input", 2: "non-manifold mesh", 3: "degenerate face"}[rc])
        self._h = h

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib is not None:
            _lib.om_mesh_free(h)
            self._h = None

    @property
    def lref(self) -> float:
        return lib().om_mesh_lref(self._h)

    def theta(self):
        t = np.zeros(len(self.X))
        b = np.zeros(len(self.X), np.uint8)
        lib().om_mesh_theta(self._h, _p(t), _p(b))
        return t, b.astype(bool)

    def adjacency(self):
        a = np.zeros((len(self.F), 3), np.int64)
        lib().om_mesh_adjacency(self._h, _p(a))
        return a


def _opts(max_steps=0, path_cap=0, tau_snap=0.0, tau_near=0.0, boundary_mode=0):
    return _Opts(max_steps, path_cap, tau_snap, tau_near, boundary_mode)


def exp_map(mesh: Mesh, face, bary, v, w=None, length=None, *, max_steps=0, tau_snap=0.0,
            tau_near=0.0, path_cap=0, boundary_mode=0, threads=0):
    """Batch exponential map (forward).  Returns a dict of numpy arrays:
    face, bary, pos, dir, w (if given), status, ncross, nvert, hash, margin, and when
    path_cap > 0 the traced geodesic: path [nq, path_cap] (faces in the order the walk enters
    them, -1 past the end), path_pt [nq, path_cap, 3] (the point where it enters each), path_len
    [nq] (faces entered, which may exceed path_cap).  tau_snap/tau_near are relative to the
    mesh's mean edge length (defaults 1e-12 and 1e-4).  boundary_mode 0 stops at the boundary
    (Sec. 4, original rule), 1 applies hole avoidance (status HOLE when it engaged)."""
    face = np.ascontiguousarray(face, dtype=np.int32)
    nq = len(face)
    bary = _f64(bary, (nq, 3))
    v = _f64(v, (nq, 3))
    nw = 0
    if w is not None:
        w = _f64(w)
        nw = w.shape[1] if w.ndim == 3 else 0
        w = w.reshape(nq, nw, 3)
        if nw == 0:
            w = None
    ln = None if length is None else _f64(length, (nq,))
    out = {
        "face": np.zeros(nq, np.int32), "bary": np.zeros((nq, 3)), "pos": np.zeros((nq, 3)),
        "dir": np.zeros((nq, 3)), "status": np.zeros(nq, np.uint32), "ncross": np.zeros(nq, np.int32),
        "nvert": np.zeros(nq, np.int32), "hash": np.zeros(nq, np.uint64), "margin": np.zeros(nq),
    }
    if nw:
        out["w"] = np.zeros((nq, nw, 3))
    if path_cap:
        out["path"] = np.zeros((nq, path_cap), np.int32)
        out["path_pt"] = np.zeros((nq, path_cap, 3))
        out["path_len"] = np.zeros(nq, np.int32)
    o = _opts(max_steps, path_cap, tau_snap, tau_near, boundary_mode)
    lib().om_exp_map(mesh._h, nq, _p(face), _p(bary), _p(v), _p(ln), nw, _p(w), _p(out["face"]),
                     _p(out["bary"]), _p(out["pos"]), _p(out["dir"]), _p(out.get("w")),
                     _p(out["status"]), _p(out["ncross"]), _p(out["nvert"]), _p(out["hash"]),
                     _p(out["margin"]), _p(out.get("path")), _p(out.get("path_pt")), _p(out.get("path_len")),
                     C.byref(o), threads)
    return out


def transport_back(mesh: Mesh, face, bary, v, u, length=None, **kw):
    """The adjoint of the parallel transport Pi along the geodesic Exp_p(v), which is its
    inverse (App. "Additional Details on Mesh-LBFGS and GCVT": the vector is moved backwards on
    the curve).  Written from the adjoint's definition <Pi a, u> = <a, Pi* u> for every tangent
    a at p: with an orthonormal basis (e1, e2) of the start face carried forward to (T1, T2),
    Pi* u = e1 <T1, u> + e2 <T2, u>.  u [nq, n_u, 3] (or [nq, 3]) at the end points.
    Returns (Pi* u in u's shape, the forward walk's output dict)."""
    face = np.ascontiguousarray(face, dtype=np.int32)
    nq = len(face)
    X, F = mesh.X, mesh.F
    x0, x1, x2 = X[F[face, 0]], X[F[face, 1]], X[F[face, 2]]
    e1 = (x1 - x0) / np.linalg.norm(x1 - x0, axis=1, keepdims=True)
    n = np.cross(x1 - x0, x2 - x0)
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    e2 = np.cross(n, e1)
    out = exp_map(mesh, face, bary, v, np.stack([e1, e2], axis=1), length, **kw)
    u = _f64(u)
    shape = u.shape
    u = u.reshape(nq, -1, 3)
    c = np.einsum("qij,qkj->qki", out["w"], u)          # <T_i, u_k>
    back = c[..., 0:1] * e1[:, None, :] + c[..., 1:2] * e2[:, None, :]
    return back.reshape(shape), out


def ep_backward(mesh: Mesh, face, bary, v, g_pos, *, threads=0, **kw):
    """Extrinsic-proxy VJP (Eq. proxy_func): grad_v; grad_p and grad_bary are zero."""
    face = np.ascontiguousarray(face, dtype=np.int32)
    nq = len(face)
    gv = np.zeros((nq, 3))
    fl = np.zeros(nq, np.uint32)
    o = _opts(**kw)
    lib().om_ep_backward(mesh._h, nq, _p(face), _p(_f64(bary, (nq, 3))), _p(_f64(v, (nq, 3))),
                         _p(_f64(g_pos, (nq, 3))), _p(gv), _p(fl), C.byref(o), threads)
    return {"grad_v": gv, "grad_p": np.zeros((nq, 3)), "grad_bary": np.zeros((nq, 3)), "flags": fl}


def gfd_backward(mesh: Mesh, face, bary, v, g_pos, eps_v=1e-4, eps_p=1e-4, *, threads=0, **kw):
    """Geodesic finite differences (Eqs. jv, jp), two batched rounds of independent walks."""
    face = np.ascontiguousarray(face, dtype=np.int32)
    nq = len(face)
    gv, gp, gb = np.zeros((nq, 3)), np.zeros((nq, 3)), np.zeros((nq, 3))
    fl = np.zeros(nq, np.uint32)
    o = _opts(**kw)
    lib().om_gfd_backward(mesh._h, nq, _p(face), _p(_f64(bary, (nq, 3))), _p(_f64(v, (nq, 3))),
                          eps_v, eps_p, _p(_f64(g_pos, (nq, 3))), _p(gv), _p(gp), _p(gb), _p(fl),
                          C.byref(o), threads)
    return {"grad_v": gv, "grad_p": gp, "grad_bary": gb, "flags": fl}


def fnv_hash(faces) -> int:
    """Word-wise FNV-1a 64 over a face sequence (the definition both sides implement)."""
    h = 0xCBF29CE484222325
    for f in faces:
        h ^= int(f) & 0xFFFFFFFF
        h = (h * 0x100000001B3) & 0xFFFFFFFFFFFFFFFF
    return h
