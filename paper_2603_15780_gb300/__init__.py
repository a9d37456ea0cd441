"""GB300-native batched straightest-geodesic exponential map (Python binding).

Thin ctypes binding over ``libsgeo.so`` (declared in ``include/sgeo.h``): argument
marshalling only.  Every step of the exponential map, the parallel transport and the
backward estimators runs in the library's CUDA kernels; PyTorch only provides device
memory, streams and ``torch.autograd.Function``.  There is no CPU fallback: if the
library cannot be loaded, or no CUDA device is present, calls raise.

    mesh = Mesh(V, F)                       # numpy float32 [N,3], int32 [F,3]
    out = exp_map(mesh, face, bary, v, w)   # torch CUDA tensors
    pos = ExpMap.apply(mesh, face, bary, v, "gfd")   # differentiable in v, bary (and V)
"""
from __future__ import annotations

import ctypes as C
import os
import threading

import numpy as np

from . import build as _build

__all__ = ["Mesh", "exp_map", "exp_map_backward", "transport_back", "ExpMap", "ExpMapFieldSteps", "exp_map_field_steps",
           "exp_map_field_steps_backward", "Opts", "lib", "status_names",
           "ST_BOUNDARY", "ST_MAX_STEPS", "ST_NEAR_VERTEX", "ST_NEAR_EDGE", "ST_VERTEX_HIT", "ST_FP64",
           "ST_START_ON_EDGE", "ST_INVALID", "ST_GFD_SPLIT", "ST_FLIPPED", "ST_NO_GRADV", "ST_HOLE", "ST_MIXED",
           "ST_REWALK_DIVERGED",
           "KERNEL_AUTO", "KERNEL_PLAIN", "KERNEL_PERSISTENT", "EST_EP", "EST_GFD", "SgError"]

ST_BOUNDARY, ST_MAX_STEPS, ST_NEAR_VERTEX, ST_NEAR_EDGE = 1, 2, 4, 8
ST_VERTEX_HIT, ST_FP64, ST_START_ON_EDGE, ST_INVALID = 16, 32, 64, 128
ST_GFD_SPLIT, ST_FLIPPED, ST_NO_GRADV = 256, 512, 1024
ST_HOLE, ST_MIXED, ST_REWALK_DIVERGED = 2048, 4096, 8192
KERNEL_AUTO, KERNEL_PLAIN, KERNEL_PERSISTENT = 0, 1, 2
EST_EP, EST_GFD = 0, 1

EXPORTED = ["sg_opts_default", "sg_status_string", "sg_mesh_create", "sg_mesh_create_batched",
            "sg_mesh_destroy", "sg_mesh_get_info", "sg_exp_map_workspace_size", "sg_exp_map",
            "sg_exp_map_backward", "sg_version", "sg_exp_map_noalloc", "sg_exp_map_backward_workspace_size",
            "sg_mesh_update_vertices", "sg_exp_map_trace", "sg_transport_back", "sg_exp_map_steps",
            "sg_exp_map_steps_backward", "sg_exp_map_steps_backward_workspace_size"]


def status_names(st: int) -> list[str]:
    names = {ST_BOUNDARY: "BOUNDARY", ST_MAX_STEPS: "MAX_STEPS", ST_NEAR_VERTEX: "NEAR_VERTEX",
             ST_NEAR_EDGE: "NEAR_EDGE", ST_VERTEX_HIT: "VERTEX_HIT", ST_FP64: "FP64",
             ST_START_ON_EDGE: "START_ON_EDGE", ST_INVALID: "INVALID", ST_GFD_SPLIT: "GFD_SPLIT",
             ST_FLIPPED: "FLIPPED", ST_NO_GRADV: "NO_GRADV", ST_HOLE: "HOLE", ST_MIXED: "MIXED",
             ST_REWALK_DIVERGED: "REWALK_DIVERGED"}
    return [n for b, n in names.items() if st & b]


class SgError(RuntimeError):
    pass


class Opts(C.Structure):
    """Mirror of sg_opts (include/sgeo.h)."""
    _fields_ = [("max_steps", C.c_int32), ("kernel", C.c_int32), ("sort", C.c_int32),
                ("block", C.c_int32), ("blocks_per_sm", C.c_int32), ("fp64_escalate", C.c_int32),
                ("tau_near", C.c_float), ("tau_snap", C.c_float), ("workspace", C.c_void_p),
                ("workspace_bytes", C.c_size_t), ("prof_events", C.c_void_p), ("boundary_mode", C.c_int32),
                ("precision", C.c_int32), ("queries_per_thread", C.c_int32), ("order", C.c_void_p)]


class MeshInfo(C.Structure):
    _fields_ = [("n_vertices", C.c_int64), ("n_faces", C.c_int64), ("n_mesh", C.c_int32),
                ("record_bytes", C.c_int32), ("device_bytes", C.c_int64), ("l_ref_mean", C.c_double),
                ("n_degenerate", C.c_int64)]


_lock = threading.Lock()
_lib = None


def lib():
    """Load libsgeo.so (building it in-tree with nvcc if it is missing or stale)."""
    global _lib
    with _lock:
        if _lib is None:
            path = _build.LIB
            if not os.path.exists(path) or os.environ.get("SGEO_REBUILD"):
                path = _build.build()
            L = C.CDLL(path)
            P = C.c_void_p
            L.sg_opts_default.argtypes = [C.POINTER(Opts)]
            L.sg_status_string.argtypes = [C.c_int]
            L.sg_status_string.restype = C.c_char_p
            L.sg_version.restype = C.c_char_p
            L.sg_mesh_create.argtypes = [P, C.c_int64, P, C.c_int64, C.POINTER(P)]
            L.sg_mesh_create_batched.argtypes = [P, P, P, P, C.c_int32, C.POINTER(P)]
            L.sg_mesh_destroy.argtypes = [P]
            L.sg_mesh_get_info.argtypes = [P, C.POINTER(MeshInfo)]
            L.sg_mesh_update_vertices.argtypes = [P, P, P]
            L.sg_exp_map_workspace_size.argtypes = [P, C.c_int64, C.POINTER(Opts), C.POINTER(C.c_size_t)]
            L.sg_exp_map.argtypes = [P, C.c_int64, P, P, P, P, P, C.c_int32, P, P, P, P, P, P, P, P, P,
                                     C.POINTER(Opts), P]
            L.sg_exp_map_noalloc.argtypes = list(L.sg_exp_map.argtypes)
            L.sg_exp_map_trace.argtypes = [P, C.c_int64, P, P, P, P, P, C.c_int32, P, P, P, P, P, P, P, P, P, P,
                                           C.POINTER(Opts), P]
            L.sg_exp_map_backward_workspace_size.argtypes = [P, C.c_int32, C.c_int64, C.c_int32,
                                                             C.POINTER(C.c_size_t)]
            L.sg_exp_map_backward.argtypes = [P, C.c_int32, C.c_float, C.c_float, C.c_int64, P, P, P, P,
                                              P, P, P, P, P, P, P, C.c_int32, P, P, P, P, P, P, P,
                                              C.POINTER(Opts), P]
            L.sg_transport_back.argtypes = [P, C.c_int64, P, P, P, P, P, P, P, C.c_int32, P, P,
                                            C.POINTER(Opts), P]
            L.sg_exp_map_steps.argtypes = [P, C.c_int32, C.c_float, P, C.c_int64, P, P, P, P, P, P, P, P,
                                           P, P, P, P, P, P, C.POINTER(Opts), P]
            L.sg_exp_map_steps_backward.argtypes = [P, C.c_int32, C.c_float, C.c_float, C.c_int32, C.c_float, P,
                                                    C.c_int64, P, P, P, P, P, P, P, P, P, P, P,
                                                    C.POINTER(Opts), P]
            L.sg_exp_map_steps_backward_workspace_size.argtypes = [P, C.c_int32, C.c_int32, C.c_int64, C.c_int32,
                                                                   C.POINTER(C.c_size_t)]
            for f in EXPORTED:
                if f not in ("sg_opts_default",):
                    getattr(L, f).restype = getattr(L, f).restype or C.c_int
            L.sg_opts_default.restype = None
            _lib = L
    return _lib


def _check(rc, what):
    if rc != 0:
        msg = lib().sg_status_string(rc).decode()
        raise SgError(f"{what}: {msg} (status {rc})")


def default_opts(**kw) -> Opts:
    o = Opts()
    lib().sg_opts_default(C.byref(o))
    for k, v in kw.items():
        if v is not None:
            setattr(o, k, v)
    return o


def _torch():
    import torch
    if not torch.cuda.is_available():
        raise SgError("a CUDA device is required (the library has no CPU path)")
    return torch


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _dev(t, dtype, shape=None):
    torch = _torch()
    if t is None:
        return None
    t = torch.as_tensor(t)
    if t.device.type != "cuda":
        t = t.to("cuda", non_blocking=True)
    t = t.to(dtype).contiguous()
    if shape is not None:
        t = t.reshape(shape)
    return t


class Mesh:
    """One mesh, or several meshes batched with CSR offsets (pass a list of (V, F)).
    Vertex positions float32 [N,3] and faces int32 [F,3], on the host or (one mesh, torch
    tensors) on the device; built synchronously on the current CUDA device by sg_mesh_create /
    sg_mesh_create_batched."""

    def __init__(self, V, F=None):
        torch = _torch()
        h = C.c_void_p()
        if F is not None and isinstance(V, torch.Tensor) and V.is_cuda:
            # device arrays go to sg_mesh_create as they are (the library copies them to the host)
            Vd = V.detach().to(torch.float32).contiguous().reshape(-1, 3)
            Fd = torch.as_tensor(F, device=Vd.device).to(torch.int32).contiguous().reshape(-1, 3)
            _check(lib().sg_mesh_create(_ptr(Vd), Vd.shape[0], _ptr(Fd), Fd.shape[0], C.byref(h)), "sg_mesh_create")
            self.n_mesh = 1
            self.v_off = np.array([0, Vd.shape[0]], np.int64)
            self.f_off = np.array([0, Fd.shape[0]], np.int64)
            self.V = Vd.cpu().numpy()
            self.F = Fd.cpu().numpy()
        elif F is not None:
            V = np.ascontiguousarray(V, dtype=np.float32).reshape(-1, 3)
            F = np.ascontiguousarray(F, dtype=np.int32).reshape(-1, 3)
            _check(lib().sg_mesh_create(V.ctypes.data_as(C.c_void_p), len(V), F.ctypes.data_as(C.c_void_p),
                                        len(F), C.byref(h)), "sg_mesh_create")
            self.n_mesh = 1
            self.v_off = np.array([0, len(V)], np.int64)
            self.f_off = np.array([0, len(F)], np.int64)
            self.V = V
            self.F = F
        else:
            meshes = list(V)
            Vs = [np.ascontiguousarray(m[0], dtype=np.float32).reshape(-1, 3) for m in meshes]
            Fs = [np.ascontiguousarray(m[1], dtype=np.int32).reshape(-1, 3) for m in meshes]
            self.v_off = np.concatenate([[0], np.cumsum([len(x) for x in Vs])]).astype(np.int64)
            self.f_off = np.concatenate([[0], np.cumsum([len(x) for x in Fs])]).astype(np.int64)
            self.V = np.ascontiguousarray(np.concatenate(Vs))
            self.F = np.ascontiguousarray(np.concatenate(Fs))
            self.n_mesh = len(meshes)
            _check(lib().sg_mesh_create_batched(self.V.ctypes.data_as(C.c_void_p),
                                                self.v_off.ctypes.data_as(C.c_void_p),
                                                self.F.ctypes.data_as(C.c_void_p),
                                                self.f_off.ctypes.data_as(C.c_void_p), self.n_mesh,
                                                C.byref(h)), "sg_mesh_create_batched")
        self._h = h
        self.n_vertices = int(self.v_off[-1])
        self.n_faces = int(self.f_off[-1])

    @property
    def handle(self):
        return self._h

    def update_vertices(self, V, stream=None):
        """Move the vertices to V (float32 [n_vertices, 3], any device; same faces) and re-derive
        the mesh geometry on the GPU with sg_mesh_update_vertices.  Enqueued on `stream` (default:
        torch's current stream).  Returns the device copy of V that the call read; it is
        recorded on the stream, so the caching allocator does not reuse it before the update ran."""
        torch = _torch()
        Vd = _dev(V, torch.float32, (-1, 3))
        if Vd.shape[0] != self.n_vertices:
            raise SgError(f"update_vertices: expected {self.n_vertices} vertices, got {Vd.shape[0]}")
        s = stream if stream is not None else torch.cuda.current_stream()
        _check(lib().sg_mesh_update_vertices(self._h, _ptr(Vd), C.c_void_p(s.cuda_stream)),
               "sg_mesh_update_vertices")
        Vd.record_stream(s)
        return Vd

    def info(self) -> MeshInfo:
        i = MeshInfo()
        _check(lib().sg_mesh_get_info(self._h, C.byref(i)), "sg_mesh_get_info")
        return i

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value and _lib is not None:
            _lib.sg_mesh_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def workspace_size(mesh: Mesh, nq: int, opts: Opts | None = None) -> int:
    n = C.c_size_t()
    _check(lib().sg_exp_map_workspace_size(mesh.handle, nq, C.byref(opts or default_opts()), C.byref(n)),
           "sg_exp_map_workspace_size")
    return n.value


def exp_map(mesh: Mesh, face, bary, v, w=None, length=None, mesh_id=None, *, want_hash=False,
            want_ncross=True, opts: Opts | None = None, workspace=None, out=None, stream=None, order=None,
            **opt_kw):
    """sg_exp_map on torch CUDA tensors.  Returns dict(face, bary, pos, dir, w, status,
    ncross, hash).  `opts` (or keyword overrides such as kernel=KERNEL_PLAIN, sort=0,
    fp64_escalate=0, block=128) map to sg_opts.  `order`: an int32 [nq] CUDA tensor that receives
    the order the queries were walked in (sg_opts.order), for exp_map_backward(order=...)."""
    torch = _torch()
    face = _dev(face, torch.int32)
    nq = face.numel()
    bary = _dev(bary, torch.float32, (nq, 3))
    v = _dev(v, torch.float32, (nq, 3))
    nw = 0
    if w is not None:
        w = _dev(w, torch.float32)
        nw = w.shape[1] if w.dim() == 3 else (w.numel() // (3 * max(nq, 1)))
        w = w.reshape(nq, nw, 3) if nw else None
    length = _dev(length, torch.float32, (nq,))
    mesh_id = _dev(mesh_id, torch.int32, (nq,))
    o = opts if opts is not None else default_opts(**opt_kw)
    if order is not None:
        o.order = _order_ptr(order, nq)
    if out is None:
        dev = face.device
        out = {"face": torch.empty(nq, dtype=torch.int32, device=dev),
               "bary": torch.empty(nq, 3, device=dev), "pos": torch.empty(nq, 3, device=dev),
               "dir": torch.empty(nq, 3, device=dev),
               "status": torch.empty(nq, dtype=torch.int32, device=dev)}
        if nw:
            out["w"] = torch.empty(nq, nw, 3, device=dev)
        if want_ncross:
            out["ncross"] = torch.empty(nq, dtype=torch.int32, device=dev)
        if want_hash:
            out["hash"] = torch.empty(nq, dtype=torch.int64, device=dev)
    if workspace is None:
        # the persistent kernel's queue and sorts, and the automatic precision's escalation list
        nb = workspace_size(mesh, nq, o)
        workspace = torch.empty(max(nb, 1), dtype=torch.uint8, device=face.device)
    if workspace is not None:
        o.workspace = workspace.data_ptr()
        o.workspace_bytes = workspace.numel()
    s = stream if stream is not None else torch.cuda.current_stream()
    rc = lib().sg_exp_map(mesh.handle, nq, _ptr(mesh_id), _ptr(face), _ptr(bary), _ptr(v), _ptr(length), nw,
                          _ptr(w), _ptr(out["face"]), _ptr(out["bary"]), _ptr(out["pos"]), _ptr(out["dir"]),
                          _ptr(out.get("w")), _ptr(out["status"]), _ptr(out.get("ncross")),
                          _ptr(out.get("hash")), C.byref(o), C.c_void_p(s.cuda_stream))
    _check(rc, "sg_exp_map")
    out["_workspace"] = workspace
    return out


def exp_map_trace(mesh: Mesh, face, bary, v, length=None, mesh_id=None, *, path_cap: int = 64,
                  want_points=True, want_hash=False, opts: Opts | None = None, workspace=None, stream=None,
                  **opt_kw):
    """sg_exp_map_trace on torch CUDA tensors: the exponential map plus the traced geodesic.
    Returns dict(face, bary, pos, dir, status, ncross, hash (if want_hash), path_face [nq, cap],
    path_pt [nq, cap, 3] (if want_points), path_len [nq]).  The polyline of query i is
    path_pt[i, :path_len[i]] followed by pos[i] when path_len[i] <= path_cap; path entries
    past path_len are not written (their contents are unspecified)."""
    torch = _torch()
    face = _dev(face, torch.int32)
    nq = face.numel()
    bary = _dev(bary, torch.float32, (nq, 3))
    v = _dev(v, torch.float32, (nq, 3))
    length = _dev(length, torch.float32, (nq,))
    mesh_id = _dev(mesh_id, torch.int32, (nq,))
    o = opts if opts is not None else default_opts(**opt_kw)
    dev = face.device
    out = {"face": torch.empty(nq, dtype=torch.int32, device=dev),
           "bary": torch.empty(nq, 3, device=dev), "pos": torch.empty(nq, 3, device=dev),
           "dir": torch.empty(nq, 3, device=dev), "status": torch.empty(nq, dtype=torch.int32, device=dev),
           "ncross": torch.empty(nq, dtype=torch.int32, device=dev),
           "path_face": torch.empty(nq, path_cap, dtype=torch.int32, device=dev),
           "path_len": torch.empty(nq, dtype=torch.int32, device=dev)}
    if want_points:
        out["path_pt"] = torch.empty(nq, path_cap, 3, device=dev)
    if want_hash:
        out["hash"] = torch.empty(nq, dtype=torch.int64, device=dev)
    if workspace is None:
        workspace = torch.empty(workspace_size(mesh, nq, o), dtype=torch.uint8, device=dev)
    o.workspace = workspace.data_ptr()
    o.workspace_bytes = workspace.numel()
    s = stream if stream is not None else torch.cuda.current_stream()
    rc = lib().sg_exp_map_trace(mesh.handle, nq, _ptr(mesh_id), _ptr(face), _ptr(bary), _ptr(v), _ptr(length),
                                path_cap, _ptr(out["path_face"]), _ptr(out.get("path_pt")), _ptr(out["path_len"]),
                                _ptr(out["face"]), _ptr(out["bary"]), _ptr(out["pos"]), _ptr(out["dir"]),
                                _ptr(out["status"]), _ptr(out["ncross"]), _ptr(out.get("hash")), C.byref(o),
                                C.c_void_p(s.cuda_stream))
    _check(rc, "sg_exp_map_trace")
    return out


def backward_workspace_size(mesh: Mesh, estimator, nq: int, want_grad_V: bool) -> int:
    est = {"ep": EST_EP, "gfd": EST_GFD}.get(estimator, estimator)
    n = C.c_size_t()
    _check(lib().sg_exp_map_backward_workspace_size(mesh.handle, est, nq, int(bool(want_grad_V)), C.byref(n)),
           "sg_exp_map_backward_workspace_size")
    return n.value


def _order_ptr(order, nq: int):
    """Device pointer of a query-order buffer (int32 [nq], contiguous, CUDA), or None."""
    if order is None:
        return None
    torch = _torch()
    if order.dtype != torch.int32 or not order.is_cuda or not order.is_contiguous() or order.numel() != nq:
        raise SgError(f"order: expected a contiguous int32 CUDA tensor of {nq} entries")
    return order.data_ptr()


def exp_map_backward(mesh: Mesh, estimator, face, bary, v, end_face, end_bary, end_dir, end_status, g_pos,
                     mesh_id=None, *, g_bary=None, g_dir=None, g_w=None, eps_v=1e-4, eps_p=1e-4,
                     want_grad_V=False, grad_V=None, opts: Opts | None = None, workspace=None, stream=None,
                     order=None):
    """sg_exp_map_backward.  estimator: "ep"/"gfd" or EST_*.  Upstream gradients: g_pos (end
    point), optional g_bary (end barycentrics), g_dir (end direction), g_w [nq, n_w, 3] (carried
    vectors).  Returns dict(grad_v, grad_p, grad_bary, grad_w (if g_w), grad_V (if requested;
    accumulated into `grad_V` when given), status)."""
    torch = _torch()
    est = {"ep": EST_EP, "gfd": EST_GFD}.get(estimator, estimator)
    face = _dev(face, torch.int32)
    nq = face.numel()
    bary = _dev(bary, torch.float32, (nq, 3))
    v = _dev(v, torch.float32, (nq, 3))
    end_face = _dev(end_face, torch.int32, (nq,))
    end_dir = _dev(end_dir, torch.float32, (nq, 3))
    end_status = _dev(end_status, torch.int32, (nq,))
    end_bary = _dev(end_bary, torch.float32, (nq, 3))
    g_pos = _dev(g_pos, torch.float32, (nq, 3))
    g_bary = _dev(g_bary, torch.float32, (nq, 3))
    g_dir = _dev(g_dir, torch.float32, (nq, 3))
    n_w = 0
    if g_w is not None:
        g_w = _dev(g_w, torch.float32)
        n_w = g_w.numel() // (3 * max(nq, 1))
        g_w = g_w.reshape(nq, n_w, 3)
    mesh_id = _dev(mesh_id, torch.int32, (nq,))
    dev = face.device
    res = {"grad_v": torch.empty(nq, 3, device=dev), "grad_p": torch.empty(nq, 3, device=dev),
           "grad_bary": torch.empty(nq, 3, device=dev),
           "status": torch.empty(nq, dtype=torch.int32, device=dev)}
    if n_w:
        res["grad_w"] = torch.empty(nq, n_w, 3, device=dev)
    if want_grad_V or grad_V is not None:
        if grad_V is None:
            grad_V = torch.zeros(mesh.n_vertices, 3, device=dev)
        res["grad_V"] = grad_V
    o = opts if opts is not None else default_opts()
    if order is not None:  # the forward call's order (else the one in opts, if any)
        o.order = _order_ptr(order, nq)
    if workspace is None:
        workspace = torch.empty(backward_workspace_size(mesh, est, nq, "grad_V" in res), dtype=torch.uint8,
                                device=dev)
    o.workspace = workspace.data_ptr()
    o.workspace_bytes = workspace.numel()
    s = stream if stream is not None else torch.cuda.current_stream()
    rc = lib().sg_exp_map_backward(mesh.handle, est, eps_v, eps_p, nq, _ptr(mesh_id), _ptr(face), _ptr(bary),
                                   _ptr(v), _ptr(end_face), _ptr(end_bary), _ptr(end_dir), _ptr(end_status),
                                   _ptr(g_pos), _ptr(g_bary), _ptr(g_dir), n_w, _ptr(g_w if n_w else None),
                                   _ptr(res["grad_v"]), _ptr(res["grad_p"]), _ptr(res["grad_bary"]),
                                   _ptr(res.get("grad_V")), _ptr(res.get("grad_w")), _ptr(res["status"]),
                                   C.byref(o), C.c_void_p(s.cuda_stream))
    _check(rc, "sg_exp_map_backward")
    return res


def transport_back(mesh: Mesh, face, bary, v, end, u, mesh_id=None, *, opts: Opts | None = None, stream=None):
    """sg_transport_back: move tangent vectors u [nq, n_u, 3] (or [nq, 3]) at the end points of
    the geodesics Exp_p(v) back to their start points, the adjoint (= inverse) of the forward
    parallel transport.  `end` is the forward's output dict (face, dir, status).  Returns a
    tensor of u's shape."""
    torch = _torch()
    face = _dev(face, torch.int32)
    nq = face.numel()
    bary = _dev(bary, torch.float32, (nq, 3))
    v = _dev(v, torch.float32, (nq, 3))
    end_face = _dev(end["face"], torch.int32, (nq,))
    end_dir = _dev(end["dir"], torch.float32, (nq, 3))
    end_status = _dev(end.get("status"), torch.int32, (nq,))
    u = _dev(u, torch.float32)
    shape = u.shape
    n_u = u.numel() // (3 * max(nq, 1))
    u = u.reshape(nq, n_u, 3)
    mesh_id = _dev(mesh_id, torch.int32, (nq,))
    out = torch.empty(nq, n_u, 3, device=face.device)
    o = opts if opts is not None else default_opts()
    s = stream if stream is not None else torch.cuda.current_stream()
    rc = lib().sg_transport_back(mesh.handle, nq, _ptr(mesh_id), _ptr(face), _ptr(bary), _ptr(v), _ptr(end_face),
                                 _ptr(end_dir), _ptr(end_status), n_u, _ptr(u), _ptr(out), C.byref(o),
                                 C.c_void_p(s.cuda_stream))
    _check(rc, "sg_transport_back")
    return out.reshape(shape)


def exp_map_field_steps(mesh: Mesh, face, bary, U, K: int, h: float | None = None, mesh_id=None, *,
                        want_steps=True, want_hash=False, opts: Opts | None = None, stream=None):
    """sg_exp_map_steps: K exponential-map steps x_{k+1} = Exp_{x_k}(h u(x_k)) of the vector field
    whose values at the vertices are U [n_vertices, 3] (barycentric interpolation inside a face), in
    one launch; h defaults to 1 / K.  Returns dict(face, bary, pos, dir, status) of the last step,
    with want_steps the per-step records step_face [K+1, nq], step_bary [K+1, nq, 3], step_v [K, nq, 3],
    step_dir [K, nq, 3], step_status [K, nq] (and step_hash [K, nq] with want_hash)."""
    torch = _torch()
    face = _dev(face, torch.int32)
    nq = face.numel()
    bary = _dev(bary, torch.float32, (nq, 3))
    U = _dev(U, torch.float32, (-1, 3))
    mesh_id = _dev(mesh_id, torch.int32, (nq,))
    h = (1.0 / K if K > 0 else 0.0) if h is None else float(h)   # K < 1 is rejected by the library
    dev = face.device
    out = {"face": torch.empty(nq, dtype=torch.int32, device=dev), "bary": torch.empty(nq, 3, device=dev),
           "pos": torch.empty(nq, 3, device=dev), "dir": torch.empty(nq, 3, device=dev),
           "status": torch.empty(nq, dtype=torch.int32, device=dev)}
    if want_steps and K > 0:
        out.update({"step_face": torch.empty(K + 1, nq, dtype=torch.int32, device=dev),
                    "step_bary": torch.empty(K + 1, nq, 3, device=dev), "step_v": torch.empty(K, nq, 3, device=dev),
                    "step_dir": torch.empty(K, nq, 3, device=dev),
                    "step_status": torch.empty(K, nq, dtype=torch.int32, device=dev)})
        if want_hash:
            out["step_hash"] = torch.empty(K, nq, dtype=torch.int64, device=dev)
    o = opts if opts is not None else default_opts()
    ws = torch.empty(64, dtype=torch.uint8, device=dev)
    o.workspace = ws.data_ptr()
    o.workspace_bytes = 64
    s = stream if stream is not None else torch.cuda.current_stream()
    rc = lib().sg_exp_map_steps(mesh.handle, K, h, _ptr(U), nq, _ptr(mesh_id), _ptr(face), _ptr(bary),
                                _ptr(out["face"]), _ptr(out["bary"]), _ptr(out["pos"]), _ptr(out["dir"]),
                                _ptr(out["status"]), _ptr(out.get("step_face")), _ptr(out.get("step_bary")),
                                _ptr(out.get("step_v")), _ptr(out.get("step_dir")), _ptr(out.get("step_status")),
                                _ptr(out.get("step_hash")), C.byref(o), C.c_void_p(s.cuda_stream))
    _check(rc, "sg_exp_map_steps")
    out["_workspace"] = ws
    return out


def exp_map_field_steps_backward(mesh: Mesh, estimator, fwd: dict, U, K: int, h: float, g_pos, g_bary=None,
                                 mesh_id=None, *, eps_v=1e-4, eps_p=1e-4, grad_U=None, want_grad_V=False,
                                 grad_V=None, opts: Opts | None = None, stream=None):
    """sg_exp_map_steps_backward on the per-step records of exp_map_field_steps.  Returns
    dict(grad_bary [nq, 3] of the start barycentrics, grad_U [n_vertices, 3] (accumulated into
    `grad_U` when given), grad_V (if requested))."""
    torch = _torch()
    est = {"ep": EST_EP, "gfd": EST_GFD}.get(estimator, estimator)
    nq = fwd["face"].numel()
    dev = fwd["face"].device
    U = _dev(U, torch.float32, (-1, 3))
    g_pos = _dev(g_pos, torch.float32, (nq, 3))
    g_bary = _dev(g_bary, torch.float32, (nq, 3))
    mesh_id = _dev(mesh_id, torch.int32, (nq,))
    res = {"grad_bary": torch.empty(nq, 3, device=dev),
           "grad_U": grad_U if grad_U is not None else torch.zeros(U.shape[0], 3, device=dev)}
    if want_grad_V or grad_V is not None:
        res["grad_V"] = grad_V if grad_V is not None else torch.zeros(mesh.n_vertices, 3, device=dev)
    n = C.c_size_t()
    _check(lib().sg_exp_map_steps_backward_workspace_size(mesh.handle, est, K, nq, int("grad_V" in res), C.byref(n)),
           "sg_exp_map_steps_backward_workspace_size")
    ws = torch.empty(max(n.value, 1), dtype=torch.uint8, device=dev)
    o = opts if opts is not None else default_opts()
    o.workspace = ws.data_ptr()
    o.workspace_bytes = ws.numel()
    s = stream if stream is not None else torch.cuda.current_stream()
    rc = lib().sg_exp_map_steps_backward(mesh.handle, est, eps_v, eps_p, K, h, _ptr(U), nq, _ptr(mesh_id),
                                         _ptr(fwd["step_face"]), _ptr(fwd["step_bary"]), _ptr(fwd["step_v"]),
                                         _ptr(fwd["step_dir"]), _ptr(fwd["step_status"]), _ptr(g_pos), _ptr(g_bary),
                                         _ptr(res["grad_U"]), _ptr(res["grad_bary"]), _ptr(res.get("grad_V")),
                                         C.byref(o), C.c_void_p(s.cuda_stream))
    _check(rc, "sg_exp_map_steps_backward")
    res["_workspace"] = ws
    return res


def _autograd_function():
    import torch

    class ExpMap(torch.autograd.Function):
        """(pos, face, bary, dir, status) = Exp_p(v) with p = (face, bary) on `mesh`.
        Differentiable outputs: pos, bary (so that the end point can start a next step) and dir;
        inputs v, bary and (through `V`, the mesh's vertex tensor, if it requires grad) the vertex
        positions.  estimator: "ep" (Eq. proxy_func, grad for bary is zero) or "gfd" (Eqs. jv, jp)."""

        @staticmethod
        def forward(ctx, mesh, face, bary, v, estimator="gfd", V=None, mesh_id=None, eps=1e-4):
            # the forward's query order is kept for the backward's re-walk (no second sort)
            order = torch.empty(face.numel(), dtype=torch.int32, device=face.device)
            out = exp_map(mesh, face, bary.detach(), v.detach(), mesh_id=mesh_id, order=order)
            ctx.mesh, ctx.estimator, ctx.eps = mesh, estimator, eps
            ctx.save_for_backward(face, bary.detach(), v.detach(), out["face"], out["bary"], out["dir"],
                                  out["status"], mesh_id if mesh_id is not None else torch.empty(0), order)
            ctx.has_V = V is not None
            ctx.mark_non_differentiable(out["face"], out["status"])
            ctx.set_materialize_grads(False)
            return out["pos"], out["face"], out["bary"], out["dir"], out["status"]

        @staticmethod
        def backward(ctx, g_pos, _gf, g_bary, g_dir, _gs):
            face, bary, v, ef, eb, ed, es, mid, order = ctx.saved_tensors
            if g_pos is None:
                g_pos = torch.zeros(face.numel(), 3, device=face.device)
            r = exp_map_backward(ctx.mesh, ctx.estimator, face, bary, v, ef, eb, ed, es, g_pos.contiguous(),
                                 mesh_id=mid if mid.numel() else None,
                                 g_bary=None if g_bary is None else g_bary.contiguous(),
                                 g_dir=None if g_dir is None else g_dir.contiguous(),
                                 eps_v=ctx.eps, eps_p=ctx.eps,
                                 want_grad_V=ctx.has_V and ctx.needs_input_grad[5], order=order)
            gV = r.get("grad_V")
            return None, None, r["grad_bary"], r["grad_v"], None, gV, None, None

    return ExpMap


def exp_map_steps(mesh: Mesh, face, bary, field, K: int, estimator="gfd", V=None, mesh_id=None, eps=1e-4,
                  x0=None, return_steps=False):
    """The K-step exponential map of the flow-matching application (Sec. 5, Eq. fmobj):
    p_{k+1} = Exp_{p_k}(field(x_k, k) / K) for k = 0..K-1, with the vector field re-evaluated at
    each intermediate point x_k so that the trajectory can turn.  `field(x, k)` maps positions
    [nq, 3] to ambient vectors [nq, 3] (projected onto each face by the walk).  Every step is one
    differentiable ExpMap call; its end (face, bary) starts the next step and carries gradients
    back through grad_bary (GFD's J^p).  x0 defaults to the start positions, taken from a
    zero-length walk (not differentiated).  Returns (pos, face, bary, status) of the last step,
    and with return_steps=True also the list of per-step dicts (face, bary, v, end_face,
    end_bary, end_dir, status; detached)."""
    torch = _torch()
    face = _dev(face, torch.int32)
    nq = face.numel()
    if x0 is None:
        x0 = exp_map(mesh, face, _dev(bary, torch.float32, (nq, 3)), torch.zeros(nq, 3, device=face.device),
                     mesh_id=mesh_id)["pos"]
    x = x0
    st = None
    steps = []
    for k in range(K):
        v = field(x, k) / K
        f_in, b_in = face, bary
        x, face, bary, d, st_k = ExpMap.apply(mesh, face, bary, v, estimator, V, mesh_id, eps)
        st = st_k if st is None else (st | st_k)
        if return_steps:
            steps.append({"face": f_in, "bary": torch.as_tensor(b_in).detach(), "v": v.detach(), "end_face": face,
                          "end_bary": bary.detach(), "end_dir": d.detach(), "status": st_k})
    return (x, face, bary, st, steps) if return_steps else (x, face, bary, st)


def _steps_autograd_function():
    import torch

    class ExpMapFieldSteps(torch.autograd.Function):
        """(pos, face, bary, dir, status) after K steps x_{k+1} = Exp_{x_k}(h u(x_k)) of the field
        with vertex values U, in one launch (sg_exp_map_steps).  Differentiable in the start
        barycentrics `bary` and in `U`; the backward chains the K steps' estimator VJPs
        (sg_exp_map_steps_backward: "ep" or "gfd", step `eps`)."""

        @staticmethod
        def forward(ctx, mesh, face, bary, U, K, h=None, estimator="gfd", mesh_id=None, eps=1e-4):
            h = 1.0 / K if h is None else float(h)
            out = exp_map_field_steps(mesh, face, bary.detach(), U.detach(), K, h, mesh_id=mesh_id)
            ctx.mesh, ctx.K, ctx.h, ctx.estimator, ctx.eps = mesh, K, h, estimator, eps
            ctx.rec = {k: out[k] for k in ("face", "step_face", "step_bary", "step_v", "step_dir", "step_status")}
            ctx.save_for_backward(U.detach(), mesh_id if mesh_id is not None else torch.empty(0))
            ctx.mark_non_differentiable(out["face"], out["status"])
            ctx.set_materialize_grads(False)
            return out["pos"], out["face"], out["bary"], out["dir"], out["status"]

        @staticmethod
        def backward(ctx, g_pos, _gf, g_bary, _gd, _gs):
            U, mid = ctx.saved_tensors
            nq = ctx.rec["face"].numel()
            if g_pos is None:
                g_pos = torch.zeros(nq, 3, device=U.device)
            r = exp_map_field_steps_backward(ctx.mesh, ctx.estimator, ctx.rec, U, ctx.K, ctx.h, g_pos.contiguous(),
                                             None if g_bary is None else g_bary.contiguous(),
                                             mesh_id=mid if mid.numel() else None, eps_v=ctx.eps, eps_p=ctx.eps)
            return None, None, r["grad_bary"], r["grad_U"], None, None, None, None, None

    return ExpMapFieldSteps


class _Lazy:
    def __init__(self, make):
        self._make = make
        self._cls = None

    def __getattr__(self, name):
        if name.startswith("_"):
            raise AttributeError(name)
        if self._cls is None:
            self._cls = self._make()
        return getattr(self._cls, name)


ExpMap = _Lazy(_autograd_function)
ExpMapFieldSteps = _Lazy(_steps_autograd_function)
