"""Thin Python binding of libdnnmg (include/dnnmg.h) over ctypes.

Argument marshalling only: every step of the correction runs in the library's
CUDA kernels.  Tensors are torch CUDA tensors (device memory and streams come
from PyTorch); the functions check dtype, device, contiguity and size, then
pass raw pointers and the current stream.  If the shared library is missing
the import fails loudly -- there is no CPU fallback.
"""

import ctypes
import os

import numpy as np
import torch

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libdnnmg.so")

F64, F32, BF16NET = 0, 1, 2
PRECISIONS = {"f64": F64, "f32": F32, "bf16": BF16NET}
_REAL = {F64: torch.float64, F32: torch.float32, BF16NET: torch.float32}
_FEAT = {F64: torch.float64, F32: torch.float32, BF16NET: torch.bfloat16}

STATUS = {0: "DNNMG_OK", 1: "DNNMG_EINVAL", 2: "DNNMG_ECUDA", 3: "DNNMG_EUNSUPPORTED", 4: "DNNMG_ENOMEM"}


class DnnmgError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class MeshDesc(ctypes.Structure):
    _fields_ = [("nxc", ctypes.c_int), ("nyc", ctypes.c_int), ("K", ctypes.c_int), ("s", ctypes.c_int),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double),
                ("obst_cx", ctypes.c_double), ("obst_cy", ctypes.c_double),
                ("obst_ax", ctypes.c_double), ("obst_ay", ctypes.c_double),
                ("solid", ctypes.POINTER(ctypes.c_ubyte)),
                ("nu", ctypes.c_double), ("k", ctypes.c_double), ("alpha0", ctypes.c_double),
                ("u_max", ctypes.c_double), ("ramp", ctypes.c_int), ("precision", ctypes.c_int)]


class MeshInfo(ctypes.Structure):
    _fields_ = [("nxc", ctypes.c_int), ("nyc", ctypes.c_int), ("nxf", ctypes.c_int), ("nyf", ctypes.c_int),
                ("K", ctypes.c_int), ("s", ctypes.c_int), ("npx", ctypes.c_int), ("npy", ctypes.c_int),
                ("Nc", ctypes.c_longlong), ("Nf", ctypes.c_longlong),
                ("pitch", ctypes.c_int), ("plane", ctypes.c_longlong), ("P", ctypes.c_int),
                ("nf", ctypes.c_int), ("nc", ctypes.c_int), ("n_in", ctypes.c_int), ("n_out", ctypes.c_int),
                ("ldx", ctypes.c_int), ("n_solid_coarse", ctypes.c_int), ("precision", ctypes.c_int),
                ("real_bytes", ctypes.c_int), ("feature_bytes", ctypes.c_int),
                ("workspace_bytes", ctypes.c_size_t)]

    def as_dict(self):
        return {name: getattr(self, name) for name, _ in self._fields_}


class MgDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int), ("levels", ctypes.c_int),
                ("lx", ctypes.c_double), ("ly", ctypes.c_double),
                ("solid", ctypes.POINTER(ctypes.c_ubyte)),
                ("nu", ctypes.c_double), ("k", ctypes.c_double), ("alpha0", ctypes.c_double),
                ("u_max", ctypes.c_double), ("ramp", ctypes.c_int), ("precision", ctypes.c_int)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"{LIB_PATH} is missing: build it with paper_2008_11520_gb300.build.build() "
                          "(or __graft_entry__.build()); there is no fallback path")
    lib = ctypes.CDLL(LIB_PATH)
    P, I, D, S = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_size_t
    sig = {
        "dnnmg_mesh_query": [ctypes.POINTER(MeshDesc), ctypes.POINTER(MeshInfo)],
        "dnnmg_mesh_create": [ctypes.POINTER(MeshDesc), ctypes.POINTER(P)],
        "dnnmg_mesh_destroy": [P],
        "dnnmg_mesh_get_info": [P, ctypes.POINTER(MeshInfo)],
        "dnnmg_mesh_maps": [P, P, P, P, P],
        "dnnmg_net_create": [I, I, I, P, P, P, I, ctypes.POINTER(P)],
        "dnnmg_net_destroy": [P],
        "dnnmg_head_params": [I],
        "dnnmg_net_create_head": [I, I, I, P, P, P, P, I, ctypes.POINTER(P)],
        "dnnmg_head_fold": [I, I, P, P, P, P],
        "dnnmg_head_backward": [I, I, P, P, P, P, P, P, P],
        "dnnmg_prolongate": [P, P, P, D, P],
        "dnnmg_patch_features": [P, P, P, D, P, P, P, P],
        "dnnmg_gru_step": [P, P, P, P, I, P],
        "dnnmg_scatter_avg": [P, P, P, P, D, P, P],
        "dnnmg_rhs_restrict": [P, P, P, P, P],
        "dnnmg_step": [P, P, P, P, P, P, P, S, D, P],
        "dnnmg_step_host": [P, P, P, P, P, P, P, S, D, P],
        "dnnmg_step_launches": [P, P],
        "dnnmg_step_timed": [P, P, P, P, P, P, P, S, D, P, I, P],
        "dnnmg_restrict": [P, P, P, P],
        "dnnmg_rhs": [P, P, P, P],
        "dnnmg_scatter_rhs": [P, P, P, D, P, P],
        "dnnmg_step_static": [P, P, P, P, P, P, D, P],
        "dnnmg_workspace_offsets": [P, ctypes.POINTER(ctypes.c_longlong), ctypes.POINTER(ctypes.c_longlong),
                                    ctypes.POINTER(ctypes.c_longlong)],
        "dnnmg_net_status": [P, ctypes.POINTER(ctypes.c_int), I],
        "dnnmg_mesh_status": [P, ctypes.POINTER(ctypes.c_int), I],
        "dnnmg_net_uses_tensor_cores": [P],
        "dnnmg_server_create": [P, I, ctypes.POINTER(P)],
        "dnnmg_server_destroy": [P],
        "dnnmg_server_admit": [P, P, ctypes.POINTER(I)],
        "dnnmg_server_release": [P, I],
        "dnnmg_server_state": [P, I, ctypes.POINTER(P)],
        "dnnmg_server_step": [P, I, ctypes.POINTER(I), ctypes.POINTER(P), ctypes.POINTER(P), ctypes.POINTER(P),
                              ctypes.POINTER(D), P],
        "dnnmg_pool_create": [I, I, ctypes.POINTER(P)],
        "dnnmg_pool_alloc": [P, I, ctypes.POINTER(I)],
        "dnnmg_pool_free": [P, I],
        "dnnmg_pool_stats": [P, ctypes.POINTER(I), ctypes.POINTER(I)],
        "dnnmg_trainer_create": [I, I, I, I, I, I, ctypes.POINTER(P)],
        "dnnmg_trainer_destroy": [P],
        "dnnmg_trainer_set_precision": [P, I],
        "dnnmg_trainer_status": [P, ctypes.POINTER(I), I],
        "dnnmg_gemm_bf16_nt": [I, I, I, P, I, P, I, P, I, I, P, P],
        "dnnmg_gru_seq_forward": [P, P, P, P, P, P, P, P],
        "dnnmg_gru_seq_state": [P, ctypes.POINTER(P)],
        "dnnmg_gru_seq_backward": [P, P, P, P, P, P, P, P, P, P],
        "dnnmg_l2_loss": [P, P, ctypes.c_longlong, I, P, P, P],
        "dnnmg_sumsq": [P, ctypes.c_longlong, P, P],
        "dnnmg_selftest_wait_timeout": [ctypes.c_longlong, ctypes.POINTER(I), ctypes.POINTER(ctypes.c_longlong)],
        "dnnmg_adam_step": [P, P, P, P, ctypes.c_longlong, I, ctypes.c_float, ctypes.c_float, ctypes.c_float,
                            ctypes.c_float, ctypes.c_float, P],
        "dnnmg_mg_create": [ctypes.POINTER(MgDesc), ctypes.POINTER(P)],
        "dnnmg_mg_destroy": [P],
        "dnnmg_mg_level": [P, I, ctypes.POINTER(I), ctypes.POINTER(I), P],
        "dnnmg_mg_defect": [P, I, P, P, D, P, P],
        "dnnmg_mg_rhs": [P, I, P, P, P],
        "dnnmg_mg_jvp": [P, I, P, P, P, P],
        "dnnmg_mg_vanka": [P, I, P, P, P, D, P],
        "dnnmg_mg_restrict": [P, I, P, P, P],
        "dnnmg_mg_prolong_add": [P, I, P, P, P],
        "dnnmg_mg_inject": [P, I, P, P, P],
        "dnnmg_mg_dot": [P, ctypes.c_longlong, P, P, P, P],
        "dnnmg_mg_axpby": [P, ctypes.c_longlong, D, P, D, P, P],
    }
    for name, args in sig.items():
        fn = getattr(lib, name)
        fn.argtypes = args
        fn.restype = ctypes.c_int
    lib.dnnmg_server_bytes.argtypes = [P, I]
    lib.dnnmg_server_bytes.restype = ctypes.c_size_t
    lib.dnnmg_pool_destroy.argtypes = [P]
    lib.dnnmg_pool_destroy.restype = None
    lib.dnnmg_static_scratch_bytes.argtypes = []
    lib.dnnmg_static_scratch_bytes.restype = ctypes.c_size_t
    lib.dnnmg_static_scratch_needed.argtypes = [P]
    lib.dnnmg_static_scratch_needed.restype = ctypes.c_size_t
    lib.dnnmg_last_error.argtypes = []
    lib.dnnmg_last_error.restype = ctypes.c_char_p
    return lib


_lib = _load()


def lib():
    """The loaded ctypes library."""
    return _lib


def _check(code):
    if code != 0:
        raise DnnmgError(code, _lib.dnnmg_last_error().decode())


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _need(t, dtype, numel, name):
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if t.numel() != numel:
        raise ValueError(f"{name} has {t.numel()} elements, {numel} expected")


def make_desc(nxc, nyc, K, s, ellipse=None, precision="f64", solid=None, lx=2.2, ly=0.41,
              nu=1e-3, k=0.01, alpha0=0.1, u_max=1.5, ramp=False):
    d = MeshDesc()
    d.nxc, d.nyc, d.K, d.s = nxc, nyc, K, s
    d.lx, d.ly = lx, ly
    cx, cy, ax, ay = ellipse if ellipse is not None else (0.0, 0.0, 0.0, 0.0)
    d.obst_cx, d.obst_cy, d.obst_ax, d.obst_ay = cx, cy, ax, ay
    d._solid_keep = None
    if solid is not None:
        arr = np.ascontiguousarray(solid, dtype=np.uint8)
        d._solid_keep = arr
        d.solid = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))
    d.nu, d.k, d.alpha0, d.u_max = nu, k, alpha0, u_max
    d.ramp = 1 if ramp else 0
    d.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
    return d


def dnnmg_mesh_query(desc):
    info = MeshInfo()
    _check(_lib.dnnmg_mesh_query(ctypes.byref(desc), ctypes.byref(info)))
    return info


class Mesh:
    """Owning wrapper of a dnnmg_mesh_t created on the current CUDA device."""

    def __init__(self, desc):
        self.desc = desc
        h = ctypes.c_void_p()
        _check(_lib.dnnmg_mesh_create(ctypes.byref(desc), ctypes.byref(h)))
        self.handle = h
        self.info = MeshInfo()
        _check(_lib.dnnmg_mesh_get_info(h, ctypes.byref(self.info)))
        self.real = _REAL[self.info.precision]
        self.feat = _FEAT[self.info.precision]

    def close(self):
        if self.handle:
            _lib.dnnmg_mesh_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # convenience allocators (device memory from torch)
    def fine(self, ncomp, device="cuda"):
        """A zeroed fine field [ncomp][plane] in the pitched layout."""
        return torch.zeros(ncomp, self.info.plane, dtype=self.real, device=device)

    def pack(self, a, device="cuda"):
        """Node-ordered values [ncomp][Nf] (x fastest) -> pitched device field [ncomp][plane]."""
        I = self.info
        t = torch.as_tensor(a)
        ncomp = t.shape[0]
        out = torch.zeros(ncomp, I.nyf + 1, I.pitch, dtype=self.real)
        out[:, :, :I.nxf + 1] = t.reshape(ncomp, I.nyf + 1, I.nxf + 1).to(self.real)
        return out.reshape(ncomp, I.plane).to(device).contiguous()

    def unpack(self, t):
        """Pitched field [ncomp][plane] -> node-ordered float64 numpy [ncomp][Nf]."""
        I = self.info
        a = t.detach().reshape(-1, I.nyf + 1, I.pitch)[:, :, :I.nxf + 1]
        return a.double().cpu().numpy().reshape(a.shape[0], -1)

    def coarse(self, ncomp=3, device="cuda"):
        return torch.zeros(ncomp, self.info.Nc, dtype=torch.float64, device=device)

    def features(self, device="cuda"):
        return torch.zeros(self.info.P, self.info.ldx, dtype=self.feat, device=device)

    def workspace(self, device="cuda"):
        return torch.empty(self.info.workspace_bytes, dtype=torch.uint8, device=device)

    def step_outputs(self, workspace):
        """Views of the network output d [P][n_out] and of v_corr [2][plane]
        that dnnmg_step leaves in its workspace (read after the step)."""
        _, od, ov = dnnmg_workspace_offsets(self)
        I, nb = self.info, self.info.real_bytes
        d = workspace[od:od + I.P * I.n_out * nb].view(self.real).view(I.P, I.n_out)
        vc = workspace[ov:ov + 2 * I.plane * nb].view(self.real).view(2, I.plane)
        return d, vc


class Net:
    """Owning wrapper of a dnnmg_net_t (weights uploaded in the given precision).
    ``head``: the parameters theta of the convolutional head (Sec. 6.2), folded
    into the output layer on the device (dnnmg_net_create_head)."""

    def __init__(self, Wx, Uh, Wfc, precision="f64", head=None):
        Wx, Uh, Wfc = (np.ascontiguousarray(a, dtype=np.float64) for a in (Wx, Uh, Wfc))
        G, n_in = Wx.shape
        H = Uh.shape[1]
        n_out = Wfc.shape[0]
        if G != 3 * H or Uh.shape != (3 * H, H) or Wfc.shape != (n_out, H):
            raise ValueError("weight shapes must be Wx [3H][n_in], Uh [3H][H], Wfc [n_out][H]")
        self.precision = PRECISIONS[precision] if isinstance(precision, str) else int(precision)
        h = ctypes.c_void_p()
        if head is None:
            _check(_lib.dnnmg_net_create(n_in, H, n_out, Wx.ctypes.data, Uh.ctypes.data, Wfc.ctypes.data,
                                         self.precision, ctypes.byref(h)))
        else:
            head = np.ascontiguousarray(head, dtype=np.float64)
            if head.shape != (head_params(n_out),):
                raise ValueError(f"head must hold {head_params(n_out)} parameters for n_out = {n_out}")
            _check(_lib.dnnmg_net_create_head(n_in, H, n_out, Wx.ctypes.data, Uh.ctypes.data, Wfc.ctypes.data,
                                              head.ctypes.data, self.precision, ctypes.byref(h)))
        self.handle = h
        self.n_in, self.H, self.n_out = n_in, H, n_out
        self.real = _REAL[self.precision]
        self.feat = _FEAT[self.precision]

    def close(self):
        if self.handle:
            _lib.dnnmg_net_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dnnmg_mesh_maps(mesh, patch_cell=None, node_flags=None, node_mult=None, stream=None):
    I = mesh.info
    if patch_cell is not None:
        _need(patch_cell, torch.int32, I.P, "patch_cell")
    if node_flags is not None:
        _need(node_flags, torch.uint8, I.plane, "node_flags")
    if node_mult is not None:
        _need(node_mult, torch.uint8, I.plane, "node_mult")
    _check(_lib.dnnmg_mesh_maps(mesh.handle, _ptr(patch_cell), _ptr(node_flags), _ptr(node_mult),
                                _stream(stream)))


def dnnmg_prolongate(mesh, xc, xf, t, stream=None):
    I = mesh.info
    _need(xc, torch.float64, 3 * I.Nc, "xc")
    _need(xf, mesh.real, 3 * I.plane, "xf")
    _check(_lib.dnnmg_prolongate(mesh.handle, _ptr(xc), _ptr(xf), float(t), _stream(stream)))


def dnnmg_patch_features(mesh, xf, bf, X, rf=None, xc=None, t=0.0, stream=None):
    """S2+S3.  Give x~ as xf [3][plane], or pass xf=None and xc [3][Nc] (with t)
    to form x~ = P xc inside the kernel."""
    I = mesh.info
    if (xf is None) == (xc is None):
        raise ValueError("give exactly one of xf and xc")
    if xf is not None:
        _need(xf, mesh.real, 3 * I.plane, "xf")
    else:
        _need(xc, torch.float64, 3 * I.Nc, "xc")
    _need(bf, mesh.real, 2 * I.plane, "bf")
    _need(X, mesh.feat, I.P * I.ldx, "X")
    if rf is not None:
        _need(rf, mesh.real, 3 * I.plane, "rf")
    _check(_lib.dnnmg_patch_features(mesh.handle, _ptr(xf), _ptr(xc), float(t), _ptr(bf), _ptr(rf), _ptr(X),
                                     _stream(stream)))


def dnnmg_gru_step(net, X, h, d, P, stream=None):
    ldx = (net.n_in + 15) // 16 * 16
    _need(X, net.feat, P * ldx, "X")
    _need(h, net.real, P * net.H, "h")
    _need(d, net.real, P * net.n_out, "d")
    _check(_lib.dnnmg_gru_step(net.handle, _ptr(X), _ptr(h), _ptr(d), int(P), _stream(stream)))


def dnnmg_scatter_avg(mesh, d, xf, vcorr, xc=None, t=0.0, stream=None):
    """S5.  Give v~ as xf [3][plane], or pass xf=None and xc [3][Nc] (with t)."""
    I = mesh.info
    if (xf is None) == (xc is None):
        raise ValueError("give exactly one of xf and xc")
    _need(d, mesh.real, I.P * I.n_out, "d")
    if xf is not None:
        _need(xf, mesh.real, 3 * I.plane, "xf")
    else:
        _need(xc, torch.float64, 3 * I.Nc, "xc")
    _need(vcorr, mesh.real, 2 * I.plane, "vcorr")
    _check(_lib.dnnmg_scatter_avg(mesh.handle, _ptr(d), _ptr(xf), _ptr(xc), float(t), _ptr(vcorr),
                                  _stream(stream)))


def dnnmg_rhs_restrict(mesh, vcorr, bf, bc, stream=None):
    I = mesh.info
    _need(vcorr, mesh.real, 2 * I.plane, "vcorr")
    _need(bf, mesh.real, 2 * I.plane, "bf")
    _need(bc, torch.float64, 3 * I.Nc, "bc")
    _check(_lib.dnnmg_rhs_restrict(mesh.handle, _ptr(vcorr), _ptr(bf), _ptr(bc), _stream(stream)))


def dnnmg_rhs(mesh, vcorr, bf, stream=None):
    I = mesh.info
    _need(vcorr, mesh.real, 2 * I.plane, "vcorr")
    _need(bf, mesh.real, 2 * I.plane, "bf")
    _check(_lib.dnnmg_rhs(mesh.handle, _ptr(vcorr), _ptr(bf), _stream(stream)))


def dnnmg_scatter_rhs(mesh, d, xc, bf, t=0.0, stream=None):
    """S5 + S6 fused: bf = Rhs(P xc + averaged d) without writing v_corr."""
    I = mesh.info
    _need(d, mesh.real, I.P * I.n_out, "d")
    _need(xc, torch.float64, 3 * I.Nc, "xc")
    _need(bf, mesh.real, 2 * I.plane, "bf")
    _check(_lib.dnnmg_scatter_rhs(mesh.handle, _ptr(d), _ptr(xc), float(t), _ptr(bf), _stream(stream)))


def dnnmg_restrict(mesh, bf, bc, stream=None):
    I = mesh.info
    _need(bf, mesh.real, 2 * I.plane, "bf")
    _need(bc, torch.float64, 3 * I.Nc, "bc")
    _check(_lib.dnnmg_restrict(mesh.handle, _ptr(bf), _ptr(bc), _stream(stream)))


def dnnmg_net_status(net, reset=False):
    """Device status word of the network (0 = no kernel wait ran out of time)."""
    st = ctypes.c_int(0)
    _check(_lib.dnnmg_net_status(net.handle, ctypes.byref(st), 1 if reset else 0))
    return st.value


def dnnmg_mesh_status(mesh, reset=False):
    """Device status word of the mesh (0 = no stencil kernel wait ran out of time)."""
    st = ctypes.c_int(0)
    _check(_lib.dnnmg_mesh_status(mesh.handle, ctypes.byref(st), 1 if reset else 0))
    return st.value


def dnnmg_net_uses_tensor_cores(net):
    return bool(_lib.dnnmg_net_uses_tensor_cores(net.handle))


def dnnmg_step(mesh, net, xc, h, bf, bc, workspace, t, stream=None):
    I = mesh.info
    _need(xc, torch.float64, 3 * I.Nc, "xc")
    _need(h, mesh.real, I.P * net.H, "h")
    _need(bf, mesh.real, 2 * I.plane, "bf")
    _need(bc, torch.float64, 3 * I.Nc, "bc")
    if workspace.dtype != torch.uint8 or not workspace.is_cuda:
        raise TypeError("workspace must be a CUDA uint8 tensor")
    _check(_lib.dnnmg_step(mesh.handle, net.handle, _ptr(xc), _ptr(h), _ptr(bf), _ptr(bc),
                           _ptr(workspace), workspace.numel(), float(t), _stream(stream)))


def dnnmg_step_timed(mesh, net, xc, h, bf, bc, workspace, t, events, stream=None):
    """dnnmg_step recording events[0] before and events[i+1] after kernel i.

    events: dnnmg_step_launches() + 1 torch.cuda.Event objects with timing
    enabled (each is recorded once here first, which creates it)."""
    I = mesh.info
    _need(xc, torch.float64, 3 * I.Nc, "xc")
    _need(h, mesh.real, I.P * net.H, "h")
    _need(bf, mesh.real, 2 * I.plane, "bf")
    _need(bc, torch.float64, 3 * I.Nc, "bc")
    if workspace.dtype != torch.uint8 or not workspace.is_cuda:
        raise TypeError("workspace must be a CUDA uint8 tensor")
    for e in events:
        if not e.cuda_event:
            e.record()
    arr = (ctypes.c_void_p * len(events))(*[e.cuda_event for e in events])
    _check(_lib.dnnmg_step_timed(mesh.handle, net.handle, _ptr(xc), _ptr(h), _ptr(bf), _ptr(bc),
                                 _ptr(workspace), workspace.numel(), float(t), arr, len(events), _stream(stream)))


def dnnmg_step_static(mesh, net, xc, h, bf, bc, t, stream=None):
    """dnnmg_step with the library's static scratch instead of a workspace (allocates nothing)."""
    I = mesh.info
    _need(xc, torch.float64, 3 * I.Nc, "xc")
    _need(h, mesh.real, I.P * net.H, "h")
    _need(bf, mesh.real, 2 * I.plane, "bf")
    _need(bc, torch.float64, 3 * I.Nc, "bc")
    _check(_lib.dnnmg_step_static(mesh.handle, net.handle, _ptr(xc), _ptr(h), _ptr(bf), _ptr(bc), float(t),
                                  _stream(stream)))


def dnnmg_static_scratch_bytes():
    return _lib.dnnmg_static_scratch_bytes()


def dnnmg_static_scratch_needed(mesh):
    return _lib.dnnmg_static_scratch_needed(mesh.handle)


def dnnmg_workspace_offsets(mesh):
    """Byte offsets (X, d, v_corr) of what dnnmg_step leaves in its workspace."""
    x, d, v = ctypes.c_longlong(), ctypes.c_longlong(), ctypes.c_longlong()
    _check(_lib.dnnmg_workspace_offsets(mesh.handle, ctypes.byref(x), ctypes.byref(d), ctypes.byref(v)))
    return x.value, d.value, v.value


def dnnmg_step_host(mesh, net, xc_host, h, bf, bc_host, workspace, t, stream=None):
    """xc_host / bc_host: CPU float64 tensors [3][Nc] (pinned for asynchronous copies)."""
    I = mesh.info
    for name, a in (("xc_host", xc_host), ("bc_host", bc_host)):
        if a.is_cuda or a.dtype != torch.float64 or not a.is_contiguous() or a.numel() != 3 * I.Nc:
            raise TypeError(f"{name} must be a contiguous CPU float64 tensor of {3 * I.Nc} elements")
    _need(h, mesh.real, I.P * net.H, "h")
    _need(bf, mesh.real, 2 * I.plane, "bf")
    _check(_lib.dnnmg_step_host(mesh.handle, net.handle, _ptr(xc_host), _ptr(h), _ptr(bf), _ptr(bc_host),
                                _ptr(workspace), workspace.numel(), float(t), _stream(stream)))


def dnnmg_step_launches(mesh, net):
    return _lib.dnnmg_step_launches(mesh.handle, net.handle)


# ---------------------------------------------------------------- serving
class RowPool:
    """Host-only row-range allocator of the server's state pool (dnnmg_pool_*)."""

    def __init__(self, capacity_rows, unit=128):
        h = ctypes.c_void_p()
        _check(_lib.dnnmg_pool_create(int(capacity_rows), int(unit), ctypes.byref(h)))
        self.handle = h

    def alloc(self, rows):
        start = ctypes.c_int()
        _check(_lib.dnnmg_pool_alloc(self.handle, int(rows), ctypes.byref(start)))
        return start.value

    def free(self, start):
        _check(_lib.dnnmg_pool_free(self.handle, int(start)))

    def stats(self):
        used, largest = ctypes.c_int(), ctypes.c_int()
        _check(_lib.dnnmg_pool_stats(self.handle, ctypes.byref(used), ctypes.byref(largest)))
        return used.value, largest.value

    def close(self):
        if self.handle:
            _lib.dnnmg_pool_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def dnnmg_server_bytes(net, max_rows):
    return _lib.dnnmg_server_bytes(net.handle, int(max_rows))


class Server:
    """Owning wrapper of a dnnmg_server_t: batched steps of admitted instances.

    admit(mesh) -> slot; step([(slot, xc, bf, bc, t), ...]) runs one step of
    each listed instance (S4 as one launch over all of them); state(slot) is
    the instance's h as a [P][H] tensor view of the server's pool.
    """

    def __init__(self, net, max_rows):
        h = ctypes.c_void_p()
        _check(_lib.dnnmg_server_create(net.handle, int(max_rows), ctypes.byref(h)))
        self.handle = h
        self.net = net
        self.meshes = {}

    def admit(self, mesh):
        slot = ctypes.c_int()
        _check(_lib.dnnmg_server_admit(self.handle, mesh.handle, ctypes.byref(slot)))
        self.meshes[slot.value] = mesh
        return slot.value

    def release(self, slot):
        _check(_lib.dnnmg_server_release(self.handle, int(slot)))
        self.meshes.pop(slot, None)

    def state(self, slot):
        p = ctypes.c_void_p()
        _check(_lib.dnnmg_server_state(self.handle, int(slot), ctypes.byref(p)))
        P, H = self.meshes[slot].info.P, self.net.H
        if P == 0:
            return torch.empty(0, H, dtype=torch.float32, device="cuda")
        return _view_f32(p.value, P * H).view(P, H)

    def step(self, items, stream=None):
        """items: (slot, xc, bf, bc, t) per instance; xc/bc [3 Nc] FP64, bf [2][plane] FP32."""
        n = len(items)
        slots = (ctypes.c_int * n)()
        xcs, bfs, bcs = (ctypes.c_void_p * n)(), (ctypes.c_void_p * n)(), (ctypes.c_void_p * n)()
        ts = (ctypes.c_double * n)()
        for i, (slot, xc, bf, bc, t) in enumerate(items):
            I = self.meshes[slot].info
            _need(xc, torch.float64, 3 * I.Nc, "xc")
            _need(bf, torch.float32, 2 * I.plane, "bf")
            _need(bc, torch.float64, 3 * I.Nc, "bc")
            slots[i], ts[i] = slot, float(t)
            xcs[i], bfs[i], bcs[i] = xc.data_ptr(), bf.data_ptr(), bc.data_ptr()
        _check(_lib.dnnmg_server_step(self.handle, n, slots, xcs, bfs, bcs, ts, _stream(stream)))

    def close(self):
        if self.handle:
            _lib.dnnmg_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _view_f32(addr, numel):
    """A float32 CUDA tensor over device memory the library owns (no copy)."""
    class _Holder:
        __cuda_array_interface__ = {"shape": (numel,), "typestr": "<f4", "data": (addr, False), "version": 2,
                                    "strides": None}
    return torch.as_tensor(_Holder(), device="cuda")


# ---------------------------------------------------------------- convolutional head
def head_params(n_out):
    """Length of the head's parameter vector for n_out outputs (0: unsupported)."""
    return int(_lib.dnnmg_head_params(int(n_out)))


def head_fold(theta, Wfc, Weff=None, stream=None):
    """W_eff [n_out][H] = the head applied to each column of W_fc (dnnmg_head_fold; FP32 device)."""
    n_out, H = Wfc.shape
    if not head_params(n_out):
        raise DnnmgError(3, f"no head for n_out = {n_out}: it must be 2 n^2, n odd, 3..9")
    _need(theta, torch.float32, head_params(n_out), "theta")
    _need(Wfc, torch.float32, n_out * H, "Wfc")
    Weff = torch.empty_like(Wfc) if Weff is None else Weff
    _need(Weff, torch.float32, n_out * H, "Weff")
    _check(_lib.dnnmg_head_fold(n_out, H, _ptr(theta), _ptr(Wfc), _ptr(Weff), _stream(stream)))
    return Weff


def head_backward(theta, Wfc, G, stream=None):
    """(d theta, d W_fc) of sum(G * W_eff) (dnnmg_head_backward; FP32 device)."""
    n_out, H = Wfc.shape
    nt = head_params(n_out)
    _need(theta, torch.float32, nt, "theta")
    _need(Wfc, torch.float32, n_out * H, "Wfc")
    _need(G, torch.float32, n_out * H, "G")
    dtheta, dW = torch.empty_like(theta), torch.empty_like(Wfc)
    work = torch.empty(H * nt, dtype=torch.float32, device=Wfc.device)
    _check(_lib.dnnmg_head_backward(n_out, H, _ptr(theta), _ptr(Wfc), _ptr(G), _ptr(dtheta), _ptr(dW), _ptr(work),
                                    _stream(stream)))
    return dtheta, dW


# ---------------------------------------------------------------- training
def gemm_bf16_nt(A, B, C, accumulate=False, status=None, stream=None):
    """C (+)= A B^T on the tensor cores: A [M][K], B [N][K] BF16 (K contiguous,
    row strides multiples of 8), C [M][N] FP32 (dnnmg_gemm_bf16_nt)."""
    M, K = A.shape
    N = B.shape[0]
    for name, t in (("A", A), ("B", B)):
        if t.dtype != torch.bfloat16 or not t.is_cuda or t.stride(1) != 1:
            raise DnnmgError(1, f"{name} must be a CUDA bfloat16 matrix with K contiguous")
    if C.dtype != torch.float32 or not C.is_cuda or C.stride(1) != 1 or tuple(C.shape) != (M, N):
        raise DnnmgError(1, "C must be a CUDA float32 [M][N] matrix")
    st = status if status is not None else torch.zeros(1, dtype=torch.int32, device=C.device)
    _check(_lib.dnnmg_gemm_bf16_nt(M, N, K, _ptr(A), A.stride(0), _ptr(B), B.stride(0), _ptr(C), C.stride(0),
                                   1 if accumulate else 0, _ptr(st), _stream(stream)))
    return st


class Trainer:
    """Owning wrapper of a dnnmg_trainer_t: the activations of one window of
    T steps of P patch rows (FP32), for dnnmg_gru_seq_forward / _backward.
    precision "f32" multiplies in FP32 on the CUDA cores, "bf16" rounds each
    product's operands to BF16 and multiplies on the tensor cores (FP32
    accumulation; the FP32 master weights are the caller's)."""

    def __init__(self, n_in, ldx, H, n_out, T, P, precision="f32"):
        h = ctypes.c_void_p()
        _check(_lib.dnnmg_trainer_create(n_in, ldx, H, n_out, T, P, ctypes.byref(h)))
        self.handle = h
        self.n_in, self.ldx, self.H, self.n_out, self.T, self.P = n_in, ldx, H, n_out, T, P
        self.precision = precision
        if precision != "f32":
            _check(_lib.dnnmg_trainer_set_precision(h, PRECISIONS[precision]))

    def status(self, reset=False):
        """Device status bits (DNNMG_DEVERR_*) of the tensor-core products."""
        st = ctypes.c_int(0)
        _check(_lib.dnnmg_trainer_status(self.handle, ctypes.byref(st), 1 if reset else 0))
        return st.value

    def close(self):
        if self.handle:
            _lib.dnnmg_trainer_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _weights(self, Wx, Uh, Wfc):
        _need(Wx, torch.float32, 3 * self.H * self.n_in, "Wx")
        _need(Uh, torch.float32, 3 * self.H * self.H, "Uh")
        _need(Wfc, torch.float32, self.n_out * self.H, "Wfc")

    def forward(self, X, h0, Wx, Uh, Wfc, D, stream=None):
        _need(X, torch.float32, self.T * self.P * self.ldx, "X")
        if h0 is not None:
            _need(h0, torch.float32, self.P * self.H, "h0")
        self._weights(Wx, Uh, Wfc)
        _need(D, torch.float32, self.T * self.P * self.n_out, "D")
        _check(_lib.dnnmg_gru_seq_forward(self.handle, _ptr(X), _ptr(h0), _ptr(Wx), _ptr(Uh), _ptr(Wfc), _ptr(D),
                                          _stream(stream)))

    def state(self):
        """h_T of the last forward as a [P][H] view (valid until the next forward)."""
        p = ctypes.c_void_p()
        _check(_lib.dnnmg_gru_seq_state(self.handle, ctypes.byref(p)))
        return _view_f32(p.value, self.P * self.H).view(self.P, self.H)

    def backward(self, dD, X, Uh, Wfc, gWx, gUh, gWfc, dh0=None, stream=None):
        _need(dD, torch.float32, self.T * self.P * self.n_out, "dD")
        _need(X, torch.float32, self.T * self.P * self.ldx, "X")
        for name, g, W in (("gWx", gWx, 3 * self.H * self.n_in), ("gUh", gUh, 3 * self.H * self.H),
                           ("gWfc", gWfc, self.n_out * self.H)):
            _need(g, torch.float32, W, name)
        if dh0 is not None:
            _need(dh0, torch.float32, self.P * self.H, "dh0")
        _check(_lib.dnnmg_gru_seq_backward(self.handle, _ptr(dD), _ptr(X), _ptr(Uh), _ptr(Wfc), _ptr(gWx),
                                           _ptr(gUh), _ptr(gWfc), _ptr(dh0), _stream(stream)))


def dnnmg_l2_loss(D, Y, P, dD=None, stream=None):
    """Loss of Sec. 6.3 (device double tensor of one element) and, optionally, dD."""
    _need(Y, torch.float32, D.numel(), "Y")
    if dD is not None:
        _need(dD, torch.float32, D.numel(), "dD")
    out = torch.empty(1, dtype=torch.float64, device=D.device)
    _check(_lib.dnnmg_l2_loss(_ptr(D), _ptr(Y), D.numel(), int(P), _ptr(dD), _ptr(out), _stream(stream)))
    return out


def dnnmg_sumsq(x, stream=None):
    out = torch.empty(1, dtype=torch.float64, device=x.device)
    _check(_lib.dnnmg_sumsq(_ptr(x), x.numel(), _ptr(out), _stream(stream)))
    return out


def dnnmg_adam_step(p, g, m, v, step, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8, alpha=0.0, stream=None):
    for name, t in (("g", g), ("m", m), ("v", v)):
        _need(t, torch.float32, p.numel(), name)
    _check(_lib.dnnmg_adam_step(_ptr(p), _ptr(g), _ptr(m), _ptr(v), p.numel(), int(step), lr, beta1, beta2, eps,
                                alpha, _stream(stream)))


def dnnmg_selftest_wait_timeout(limit_ns):
    """Run the bounded-wait self-test; returns (status word, [thread 0 wait ns, last thread wait ns])."""
    st = ctypes.c_int()
    w = (ctypes.c_longlong * 2)()
    _check(_lib.dnnmg_selftest_wait_timeout(int(limit_ns), ctypes.byref(st), w))
    return st.value, [w[0], w[1]]



# ---------------------------------------------------------------- plain multigrid
class MG:
    """Owning wrapper of a dnnmg_mg_t: the level hierarchy of the plain
    multigrid fine solve (dnnmg_mg_* calls; iterations in mg.py)."""

    def __init__(self, nx, ny, levels, solid=None, precision="f64", lx=2.2, ly=0.41, nu=1e-3, k=0.01,
                 alpha0=0.1, u_max=1.5, ramp=False):
        d = MgDesc()
        d.nx, d.ny, d.levels = nx, ny, levels
        d.lx, d.ly, d.nu, d.k, d.alpha0, d.u_max, d.ramp = lx, ly, nu, k, alpha0, u_max, int(ramp)
        d.precision = PRECISIONS[precision]
        if d.precision == BF16NET:
            raise ValueError("the multigrid solve runs in f64 or f32")
        keep = None
        if solid is not None:
            keep = np.ascontiguousarray(np.asarray(solid, dtype=np.uint8))
            if keep.shape != (ny, nx):
                raise ValueError("solid must be [ny][nx]")
            d.solid = keep.ctypes.data_as(ctypes.POINTER(ctypes.c_ubyte))
        h = ctypes.c_void_p()
        _check(_lib.dnnmg_mg_create(ctypes.byref(d), ctypes.byref(h)))
        self.handle = h
        self.levels = levels
        self.precision = precision
        self.real = _REAL[d.precision]
        self.params = dict(lx=lx, ly=ly, nu=nu, k=k, alpha0=alpha0, u_max=u_max, ramp=ramp)

    def close(self):
        if self.handle:
            _lib.dnnmg_mg_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def level(self, l):
        """(nx, ny, solid [ny][nx] bool) of level l."""
        nx, ny = ctypes.c_int(), ctypes.c_int()
        _check(_lib.dnnmg_mg_level(self.handle, l, ctypes.byref(nx), ctypes.byref(ny), None))
        m = np.zeros((ny.value, nx.value), dtype=np.uint8)
        _check(_lib.dnnmg_mg_level(self.handle, l, None, None, m.ctypes.data_as(ctypes.c_void_p)))
        return nx.value, ny.value, m.astype(bool)

    def nodes(self, l):
        nx, ny, _ = self.level(l)
        return (nx + 1) * (ny + 1)

    def field(self, l, device="cuda"):
        return torch.zeros(3, self.nodes(l), dtype=self.real, device=device)

    def _f(self, l, t, name):
        _need(t, self.real, 3 * self.nodes(l), name)
        return _ptr(t)

    def defect(self, l, x, b, t, F, stream=None):
        _check(_lib.dnnmg_mg_defect(self.handle, l, self._f(l, x, "x"), self._f(l, b, "b"), float(t),
                                    self._f(l, F, "F"), _stream(stream)))

    def rhs(self, l, x, b, stream=None):
        _check(_lib.dnnmg_mg_rhs(self.handle, l, self._f(l, x, "x"), self._f(l, b, "b"), _stream(stream)))

    def jvp(self, l, x, dx, y, stream=None):
        _check(_lib.dnnmg_mg_jvp(self.handle, l, self._f(l, x, "x"), self._f(l, dx, "dx"), self._f(l, y, "y"),
                                 _stream(stream)))

    def vanka(self, l, x, r, dx, omega, stream=None):
        _check(_lib.dnnmg_mg_vanka(self.handle, l, self._f(l, x, "x"), self._f(l, r, "r"), self._f(l, dx, "dx"),
                                   float(omega), _stream(stream)))

    def restrict(self, l, rf, rc, stream=None):
        _check(_lib.dnnmg_mg_restrict(self.handle, l, self._f(l, rf, "rf"), self._f(l + 1, rc, "rc"),
                                      _stream(stream)))

    def prolong_add(self, l, dc, df, stream=None):
        _check(_lib.dnnmg_mg_prolong_add(self.handle, l, self._f(l + 1, dc, "dc"), self._f(l, df, "df"),
                                         _stream(stream)))

    def inject(self, l, xf, xc, stream=None):
        _check(_lib.dnnmg_mg_inject(self.handle, l, self._f(l, xf, "xf"), self._f(l + 1, xc, "xc"),
                                    _stream(stream)))

    def dot(self, a, b, out, stream=None):
        """out: a CUDA float64 tensor of one element (written on the stream)."""
        if a.dtype != self.real or b.dtype != self.real or a.numel() != b.numel():
            raise TypeError("dot: operands of the handle's precision and equal size")
        _need(out, torch.float64, 1, "out")
        _check(_lib.dnnmg_mg_dot(self.handle, a.numel(), _ptr(a), _ptr(b), _ptr(out), _stream(stream)))

    def axpby(self, alpha, x, beta, y, stream=None):
        if x.dtype != self.real or y.dtype != self.real or x.numel() != y.numel():
            raise TypeError("axpby: operands of the handle's precision and equal size")
        _check(_lib.dnnmg_mg_axpby(self.handle, x.numel(), float(alpha), _ptr(x), float(beta), _ptr(y),
                                   _stream(stream)))
