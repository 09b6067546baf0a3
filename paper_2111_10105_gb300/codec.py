"""Python binding of libmesh_codec (include/mesh_codec.h).

Argument marshalling only: every step of the codec runs in the library's
CUDA kernels.  PyTorch provides device memory and streams; there is no CPU
fallback, and importing this module fails loudly when the library has not
been built.
"""

import ctypes
import os

import numpy as np

from . import build as _build

# ---------------------------------------------------------------- ABI mirror
MC_OK = 0
STATUS_NAMES = {
    0: "MC_OK", 1: "MC_E_INVALID_ARG", 2: "MC_E_BAD_MESH", 3: "MC_E_ISOLATED_VERTEX",
    4: "MC_E_OOM", 5: "MC_E_CUDA", 6: "MC_E_NOT_CONVERGED", 7: "MC_E_BITSTREAM_CORRUPT",
    8: "MC_E_BUFFER_TOO_SMALL", 9: "MC_E_NUMERICAL", 10: "MC_E_BAD_ANCHORS",
    11: "MC_E_NO_ANCHOR_IN_COMPONENT", 12: "MC_E_TIMEOUT",
}
MC_LAYOUT_FRAMES = 0
MC_LAYOUT_VERTEX_MAJOR = 1
MC_PRECISION_FP64 = 0
MC_PRECISION_TF32 = 1
MC_PRECISION_BF16 = 2
MC_SOLVE_FRAMES = 0
MC_SOLVE_FACTORED = 1
MC_SOLVE_AUTO = 2

BUF_ROW_PTR, BUF_COL_IDX, BUF_DEGREE, BUF_ANCHORS = 0, 1, 2, 3
BUF_DELTA, BUF_BASIS, BUF_RITZ, BUF_COEFF, BUF_START = 4, 5, 6, 7, 8
BUF_DELTA_REC, BUF_CG_ITERS = 9, 10


class Params(ctypes.Structure):
    _fields_ = [
        ("n_vertices", ctypes.c_int32), ("n_triangles", ctypes.c_int32),
        ("n_frames", ctypes.c_int32), ("rank", ctypes.c_int32),
        ("coeff_bits", ctypes.c_int32), ("dict_bits", ctypes.c_int32),
        ("anchor_bits", ctypes.c_int32), ("n_anchors", ctypes.c_int32),
        ("laplacian_kind", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("oi_sweeps", ctypes.c_int32), ("cg_max_iters", ctypes.c_int32),
        ("oi_tol", ctypes.c_double), ("cg_rtol", ctypes.c_double),
        ("seed", ctypes.c_uint64), ("solve_mode", ctypes.c_int32),
        ("oi_refine_sweeps", ctypes.c_int32), ("autotune", ctypes.c_int32),
        ("block_delta", ctypes.c_int32), ("block_delta_bits", ctypes.c_int32),
        ("refine", ctypes.c_int32), ("layout", ctypes.c_int32),
        ("block_cg", ctypes.c_int32),
    ]


class Stats(ctypes.Structure):
    _fields_ = [
        ("oi_sweeps", ctypes.c_int32 * 3), ("cg_iters_max", ctypes.c_int32),
        ("cg_iters_min", ctypes.c_int32), ("cg_columns", ctypes.c_int32),
        ("cg_not_converged", ctypes.c_int32), ("cg_iterations_run", ctypes.c_int32),
        ("oi_change", ctypes.c_double * 3), ("cg_iters_mean", ctypes.c_double),
        ("cg_rel_residual_max", ctypes.c_double), ("launches_create", ctypes.c_uint64),
        ("launches_encode", ctypes.c_uint64), ("launches_decode", ctypes.c_uint64),
        ("workspace_bytes", ctypes.c_uint64),
    ]

    def as_dict(self):
        out = {}
        for name, _ in self._fields_:
            v = getattr(self, name)
            out[name] = list(v) if isinstance(v, ctypes.Array) else v
        return out


class Profile(ctypes.Structure):
    _fields_ = [
        ("n_kernels", ctypes.c_int32), ("reserved", ctypes.c_int32),
        ("name", (ctypes.c_char * 32) * 8), ("launches_timed", ctypes.c_int64 * 8),
        ("total_ms", ctypes.c_double * 8),
    ]


class MeshCodecError(RuntimeError):
    def __init__(self, status, where):
        self.status = status
        self.name = STATUS_NAMES.get(status, str(status))
        super().__init__(f"{where}: {self.name} ({status})")


_LIB = None

_P = ctypes.c_void_p
_SIGS = {
    "mesh_codec_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "mesh_codec_default_params": (None, [ctypes.POINTER(Params)]),
    "mesh_codec_create": (ctypes.c_int, [ctypes.POINTER(Params), _P, ctypes.c_int, _P,
                                         ctypes.c_int, _P, ctypes.POINTER(_P)]),
    "mesh_codec_encoded_size": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_size_t)]),
    "mesh_codec_encode": (ctypes.c_int, [_P, _P, _P, ctypes.c_size_t,
                                         ctypes.POINTER(ctypes.c_size_t), _P]),
    "mesh_codec_decode": (ctypes.c_int, [_P, _P, ctypes.c_size_t, _P, _P]),
    "mesh_codec_decode_ex": (ctypes.c_int, [_P, _P, ctypes.c_size_t, _P, _P, _P]),
    "mesh_codec_set_start_basis": (ctypes.c_int, [_P, _P, _P]),
    "mesh_codec_decode_stage": (ctypes.c_int, [_P, _P, ctypes.c_size_t, _P, _P, _P]),
    "mesh_codec_blocks_size": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t)]),
    "mesh_codec_encode_blocks": (ctypes.c_int, [_P, _P, ctypes.c_int, _P, ctypes.c_size_t,
                                                ctypes.POINTER(ctypes.c_size_t), _P]),
    "mesh_codec_decode_blocks": (ctypes.c_int, [_P, _P, ctypes.c_size_t, _P, _P]),
    "mesh_codec_rates": (ctypes.c_int, [ctypes.POINTER(Params), ctypes.c_int, _P]),
    "mesh_codec_mlp_create": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                             ctypes.c_uint64, ctypes.POINTER(_P)]),
    "mesh_codec_mlp_param_count": (ctypes.c_size_t, [_P]),
    "mesh_codec_mlp_get_params": (ctypes.c_int, [_P, ctypes.c_int, _P, _P]),
    "mesh_codec_mlp_set_params": (ctypes.c_int, [_P, _P, _P]),
    "mesh_codec_mlp_forward": (ctypes.c_int, [_P, _P, ctypes.c_longlong, _P, _P]),
    "mesh_codec_mlp_infer": (ctypes.c_int, [_P, _P, ctypes.c_longlong, _P, _P]),
    "mesh_codec_mlp_train_step": (ctypes.c_int, [_P, _P, _P, ctypes.c_longlong, ctypes.c_float,
                                                 ctypes.c_int, ctypes.POINTER(ctypes.c_double),
                                                 _P]),
    "mesh_codec_mlp_set_check_mode": (ctypes.c_int, [_P, ctypes.c_int]),
    "mesh_codec_mlp_fit_normalizer": (ctypes.c_int, [_P, _P, ctypes.c_longlong, _P]),
    "mesh_codec_mlp_get_normalizer": (ctypes.c_int, [_P, _P, _P, _P]),
    "mesh_codec_mlp_destroy": (None, [_P]),
    "mesh_codec_farthest_anchors": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P, ctypes.c_int,
                                                   _P, _P]),
    "mesh_codec_nearest_anchor": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P, _P, _P, _P,
                                                 _P]),
    "mesh_codec_warm_features": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, _P, _P,
                                                _P, _P, _P, _P, _P, ctypes.c_float, _P, _P, _P,
                                                _P]),
    "mesh_codec_warm_compose": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P, _P, _P, _P]),
    "mesh_codec_sample_rows": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_longlong, ctypes.c_uint64,
                                              ctypes.c_longlong, _P, _P]),
    "mesh_codec_basis_features": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P, _P, _P, _P, _P]),
    "mesh_codec_basis_compose": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, _P, _P, _P, _P]),
    "mesh_codec_encode_host": (ctypes.c_int, [_P, _P, _P, ctypes.c_size_t,
                                              ctypes.POINTER(ctypes.c_size_t), _P]),
    "mesh_codec_decode_host": (ctypes.c_int, [_P, _P, ctypes.c_size_t, _P, _P]),
    "mesh_codec_get_stats": (ctypes.c_int, [_P, ctypes.POINTER(Stats)]),
    "mesh_codec_buffer_size": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_size_t),
                                              ctypes.POINTER(ctypes.c_size_t)]),
    "mesh_codec_copy_buffer": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_size_t, _P]),
    "mesh_codec_set_profiling": (ctypes.c_int, [_P, ctypes.c_int]),
    "mesh_codec_get_profile": (ctypes.c_int, [_P, ctypes.POINTER(Profile)]),
    "mesh_codec_destroy": (None, [_P]),
    "mesh_codec_selftest_gemm": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                                ctypes.c_int, ctypes.c_int, _P, _P, _P, _P]),
    "mesh_codec_set_wait_limit": (ctypes.c_int, [ctypes.c_ulonglong]),
    "mesh_codec_encode_batch": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, _P, _P, _P]),
    "mesh_codec_decode_batch": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, _P, _P]),
    "mesh_codec_decode_batch_ex": (ctypes.c_int, [_P, ctypes.c_int, _P, _P, _P, _P, ctypes.c_int,
                                                  _P]),
    "mesh_codec_adjacency_static": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_int, _P, _P,
                                                   ctypes.c_size_t, _P,
                                                   ctypes.POINTER(ctypes.c_int32), _P]),
}


def library_path():
    return _build.LIB


def load_library(build_if_missing=False):
    """Load libmesh_codec.so (building it first when asked).  Raises
    ImportError when the library is absent: there is no fallback path."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if build_if_missing and not os.path.exists(path):
        _build.build()
    if not os.path.exists(path):
        raise ImportError(f"libmesh_codec.so not built ({path}); run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _LIB = lib
    return lib


def default_params():
    p = Params()
    load_library().mesh_codec_default_params(ctypes.byref(p))
    return p


def _check(status, where):
    if status != MC_OK:
        raise MeshCodecError(status, where)


def _torch():
    import torch  # noqa: WPS433  (device memory and streams only)
    return torch


def _stream_ptr(stream):
    torch = _torch()
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


class MeshCodec:
    """One codec handle for a fixed connectivity (see mesh_codec_create).

    tris: int32 [T, 3] (numpy or a CUDA tensor).  Keyword arguments set
    fields of mesh_codec_params_t (n_frames, rank, n_anchors, coeff_bits, ...).
    """

    def __init__(self, tris, n_vertices, anchors=None, stream=None, **kw):
        torch = _torch()
        lib = load_library()
        p = default_params()
        p.n_vertices = int(n_vertices)
        p.n_triangles = int(tris.shape[0])
        for key, val in kw.items():
            if not hasattr(p, key):
                raise TypeError(f"unknown parameter {key}")
            setattr(p, key, val)
        self.params = p
        if isinstance(tris, np.ndarray):
            tri_t = torch.from_numpy(np.ascontiguousarray(tris, dtype=np.int32)).cuda()
        else:
            tri_t = tris.to(device="cuda", dtype=torch.int32).contiguous()
        anc_ptr = None
        self._anc_t = None
        if anchors is not None:
            if isinstance(anchors, torch.Tensor):
                self._anc_t = anchors.to(device="cuda", dtype=torch.int32).contiguous()
            else:
                self._anc_t = torch.as_tensor(np.asarray(anchors, dtype=np.int32)).cuda()
            anc_ptr = ctypes.c_void_p(self._anc_t.data_ptr())
        h = ctypes.c_void_p()
        st = lib.mesh_codec_create(ctypes.byref(p), ctypes.c_void_p(tri_t.data_ptr()), 1, anc_ptr,
                                   1, _stream_ptr(stream), ctypes.byref(h))
        _check(st, "mesh_codec_create")
        self._h = h
        self._lib = lib
        size = ctypes.c_size_t()
        _check(lib.mesh_codec_encoded_size(h, ctypes.byref(size)), "mesh_codec_encoded_size")
        self.stream_bytes = size.value
        self.n, self.F, self.k = p.n_vertices, p.n_frames, p.rank
        # positions at the boundary: [F, n, 3], or [n, 3, F] vertex-major
        self.pos_shape = ((self.n, 3, self.F) if p.layout == MC_LAYOUT_VERTEX_MAJOR
                          else (self.F, self.n, 3))

    # ------------------------------------------------------------ device API
    def encode(self, positions, out=None, stream=None):
        """positions: CUDA float64 [F, n, 3] ([n, 3, F] with the vertex-major
        layout) -> CUDA uint8 bitstream."""
        torch = _torch()
        assert positions.is_cuda and positions.dtype == torch.float64
        assert tuple(positions.shape) == self.pos_shape and positions.is_contiguous()
        if out is None:
            out = torch.empty(self.stream_bytes, dtype=torch.uint8, device=positions.device)
        written = ctypes.c_size_t()
        st = self._lib.mesh_codec_encode(self._h, ctypes.c_void_p(positions.data_ptr()),
                                         ctypes.c_void_p(out.data_ptr()), out.numel(),
                                         ctypes.byref(written), _stream_ptr(stream))
        _check(st, "mesh_codec_encode")
        return out[: written.value]

    def decode(self, bitstream, out=None, stream=None, allow_not_converged=False, x0=None):
        """bitstream: CUDA uint8 -> CUDA float64 [F, n, 3].  x0 (CUDA float64
        [F, n, 3], frames solve only) is the CG's first iterate."""
        torch = _torch()
        assert bitstream.is_cuda and bitstream.dtype == torch.uint8
        if out is None:
            out = torch.empty(self.pos_shape, dtype=torch.float64, device=bitstream.device)
        x0p = None
        if x0 is not None:
            assert x0.is_cuda and x0.dtype == torch.float64 and x0.is_contiguous()
            assert tuple(x0.shape) == self.pos_shape
            x0p = ctypes.c_void_p(x0.data_ptr())
        st = self._lib.mesh_codec_decode_ex(self._h, ctypes.c_void_p(bitstream.data_ptr()),
                                            bitstream.numel(), x0p,
                                            ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream))
        if not (allow_not_converged and st == 6):
            _check(st, "mesh_codec_decode")
        return out

    def decode_stage(self, bitstream, stream=None):
        """Unpack + back-projection only: (delta~ [n, 3F] vertex-major,
        dequantized anchor positions [3, n_c, F]) as CUDA float64 tensors."""
        torch = _torch()
        assert bitstream.is_cuda and bitstream.dtype == torch.uint8
        n_c = self.params.n_anchors
        delta = torch.empty((self.n, 3 * self.F), dtype=torch.float64, device=bitstream.device)
        anc = torch.empty((3, max(n_c, 1), self.F), dtype=torch.float64, device=bitstream.device)
        st = self._lib.mesh_codec_decode_stage(self._h, ctypes.c_void_p(bitstream.data_ptr()),
                                               bitstream.numel(), ctypes.c_void_p(delta.data_ptr()),
                                               ctypes.c_void_p(anc.data_ptr()), _stream_ptr(stream))
        _check(st, "mesh_codec_decode_stage")
        return delta, anc[:, :n_c]

    # ------------------------------------------------------------ blocks variant
    def blocks_size(self, n_blocks):
        size = ctypes.c_size_t()
        _check(self._lib.mesh_codec_blocks_size(self._h, int(n_blocks), ctypes.byref(size)),
               "mesh_codec_blocks_size")
        return size.value

    def encode_blocks(self, positions, n_blocks, out=None, stream=None):
        """positions: CUDA float64 [n_blocks * F, n, 3] -> CUDA uint8 container
        (Section III-A: block 1 from the eigendecomposition of R[1], blocks
        2..n_b from Algorithm 1's sweeps started at the previous basis)."""
        torch = _torch()
        assert positions.is_cuda and positions.dtype == torch.float64
        assert tuple(positions.shape) == (n_blocks * self.F, self.n, 3)
        assert positions.is_contiguous()
        total = self.blocks_size(n_blocks)
        if out is None:
            out = torch.empty(total, dtype=torch.uint8, device=positions.device)
        written = ctypes.c_size_t()
        st = self._lib.mesh_codec_encode_blocks(self._h, ctypes.c_void_p(positions.data_ptr()),
                                                int(n_blocks), ctypes.c_void_p(out.data_ptr()),
                                                out.numel(), ctypes.byref(written),
                                                _stream_ptr(stream))
        _check(st, "mesh_codec_encode_blocks")
        return out[: written.value]

    def decode_blocks(self, container, n_blocks, out=None, stream=None, allow_not_converged=False):
        """Container of encode_blocks -> CUDA float64 [n_blocks * F, n, 3]."""
        torch = _torch()
        assert container.is_cuda and container.dtype == torch.uint8
        if out is None:
            out = torch.empty((n_blocks * self.F, self.n, 3), dtype=torch.float64,
                              device=container.device)
        st = self._lib.mesh_codec_decode_blocks(self._h, ctypes.c_void_p(container.data_ptr()),
                                                container.numel(), ctypes.c_void_p(out.data_ptr()),
                                                _stream_ptr(stream))
        if not (allow_not_converged and st == 6):
            _check(st, "mesh_codec_decode_blocks")
        return out

    def set_start_basis(self, q0=None, stream=None):
        """Orthogonal-iteration start basis: CUDA float64 [3, F, k] (made
        orthonormal), or None for the seeded random start."""
        ptr = None
        if q0 is not None:
            torch = _torch()
            assert q0.is_cuda and q0.dtype == torch.float64 and q0.is_contiguous()
            assert tuple(q0.shape) == (3, self.F, self.k)
            ptr = ctypes.c_void_p(q0.data_ptr())
        _check(self._lib.mesh_codec_set_start_basis(self._h, ptr, _stream_ptr(stream)),
               "mesh_codec_set_start_basis")

    # ------------------------------------------------------------ host API
    def encode_host(self, positions, out=None, stream=None):
        """positions: numpy / pinned CPU tensor float64 [F, n, 3] -> host bytes."""
        ptr, keep = _host_ptr(positions, np.float64, self.pos_shape)
        if out is None:
            out = np.empty(self.stream_bytes, dtype=np.uint8)
        optr, okeep = _host_ptr(out, np.uint8, None)
        written = ctypes.c_size_t()
        st = self._lib.mesh_codec_encode_host(self._h, ptr, optr, self.stream_bytes,
                                              ctypes.byref(written), _stream_ptr(stream))
        _check(st, "mesh_codec_encode_host")
        del keep, okeep
        return out

    def decode_host(self, bitstream, out=None, stream=None):
        ptr, keep = _host_ptr(bitstream, np.uint8, None)
        if out is None:
            out = np.empty(self.pos_shape, dtype=np.float64)
        optr, okeep = _host_ptr(out, np.float64, self.pos_shape)
        nbytes = bitstream.numel() if hasattr(bitstream, "numel") else len(bitstream)
        st = self._lib.mesh_codec_decode_host(self._h, ptr, nbytes, optr, _stream_ptr(stream))
        _check(st, "mesh_codec_decode_host")
        del keep, okeep
        return out

    # ------------------------------------------------------------ inspection
    def stats(self):
        s = Stats()
        _check(self._lib.mesh_codec_get_stats(self._h, ctypes.byref(s)), "mesh_codec_get_stats")
        return s.as_dict()

    def set_profiling(self, every):
        """Time the decoder's CG kernels with CUDA events on every `every`-th
        iteration (0 = off); resets the totals."""
        _check(self._lib.mesh_codec_set_profiling(self._h, int(every)), "mesh_codec_set_profiling")

    def profile(self):
        """{kernel name: (launches timed, total ms)}"""
        p = Profile()
        _check(self._lib.mesh_codec_get_profile(self._h, ctypes.byref(p)), "mesh_codec_get_profile")
        return {bytes(p.name[i]).split(b"\0")[0].decode(): (p.launches_timed[i], p.total_ms[i])
                for i in range(p.n_kernels)}

    def buffer(self, which, stream=None):
        torch = _torch()
        cnt, eb = ctypes.c_size_t(), ctypes.c_size_t()
        _check(self._lib.mesh_codec_buffer_size(self._h, which, ctypes.byref(cnt), ctypes.byref(eb)),
               "mesh_codec_buffer_size")
        dt = {4: torch.int32, 8: torch.float64}[eb.value]
        out = torch.empty(max(cnt.value, 1), dtype=dt, device="cuda")
        _check(self._lib.mesh_codec_copy_buffer(self._h, which, ctypes.c_void_p(out.data_ptr()),
                                                cnt.value, _stream_ptr(stream)),
               "mesh_codec_copy_buffer")
        return out[: cnt.value]

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mesh_codec_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()


def _host_ptr(obj, dtype, shape):
    if isinstance(obj, np.ndarray):
        a = obj
        if a.dtype != dtype or not a.flags["C_CONTIGUOUS"]:
            raise ValueError("host buffer must be C-contiguous with the right dtype")
        if shape is not None and a.shape != shape:
            raise ValueError(f"host buffer shape {a.shape} != {shape}")
        return ctypes.c_void_p(a.ctypes.data), a
    torch = _torch()
    if isinstance(obj, torch.Tensor) and obj.device.type == "cpu":
        if not obj.is_contiguous():
            raise ValueError("host tensor must be contiguous")
        return ctypes.c_void_p(obj.data_ptr()), obj
    if isinstance(obj, (bytes, bytearray)):
        a = np.frombuffer(obj, dtype=np.uint8)
        return ctypes.c_void_p(a.ctypes.data), a
    raise TypeError("unsupported host buffer")


def selftest_gemm(kind, A, B, splits=1, stream=None):
    """C = A B^T on the tensor cores (kind 0: TF32, 1: BF16 operands, FP32
    accumulation per K split, FP64 sum of splits).  A, B: CUDA float32
    [M, K] and [N, K]."""
    torch = _torch()
    lib = load_library()
    A = A.contiguous()
    B = B.contiguous()
    M, K = A.shape
    N = B.shape[0]
    C = torch.empty((M, N), dtype=torch.float64, device=A.device)
    _check(lib.mesh_codec_selftest_gemm(int(kind), M, N, K, int(splits),
                                        ctypes.c_void_p(A.data_ptr()),
                                        ctypes.c_void_p(B.data_ptr()),
                                        ctypes.c_void_p(C.data_ptr()), _stream_ptr(stream)),
           "mesh_codec_selftest_gemm")
    return C


def set_wait_limit(ns=0):
    """Limit (GPU global-timer nanoseconds) of every wait inside the
    tensor-core kernels, process-wide; 0 restores the default (2 s)."""
    _check(load_library().mesh_codec_set_wait_limit(int(ns)), "mesh_codec_set_wait_limit")


def _ptr_array(ptrs, ctype=ctypes.c_void_p):
    arr = (ctype * len(ptrs))()
    for i, p in enumerate(ptrs):
        arr[i] = p
    return arr


def encode_batch(codecs, positions, outs=None, stream=None):
    """Encode several sequences at once (mesh_codec_encode_batch): one codec
    per sequence, positions CUDA float64 [F_i, n_i, 3].  Returns the list of
    bitstreams (CUDA uint8 views)."""
    torch = _torch()
    lib = load_library()
    count = len(codecs)
    if outs is None:
        outs = [torch.empty(c.stream_bytes, dtype=torch.uint8, device="cuda") for c in codecs]
    hs = _ptr_array([c._h.value for c in codecs])
    ps = _ptr_array([p.data_ptr() for p in positions])
    bs = _ptr_array([o.data_ptr() for o in outs])
    caps = _ptr_array([o.numel() for o in outs], ctypes.c_size_t)
    written = (ctypes.c_size_t * count)()
    sts = (ctypes.c_int * count)()
    st = lib.mesh_codec_encode_batch(ctypes.cast(hs, _P), count, ctypes.cast(ps, _P),
                                     ctypes.cast(bs, _P), ctypes.cast(caps, _P),
                                     ctypes.cast(written, _P), ctypes.cast(sts, _P),
                                     _stream_ptr(stream))
    _check(st, "mesh_codec_encode_batch")
    return [o[: written[i]] for i, o in enumerate(outs)]


MC_BATCH_GROUPED = 1


def decode_batch(codecs, bitstreams, outs=None, stream=None, allow_not_converged=False,
                 grouped=False):
    """Decode several sequences at once (mesh_codec_decode_batch_ex): every
    sequence's CG on its own stream, or with grouped the FP32 solves as
    grouped work-table batches."""
    torch = _torch()
    lib = load_library()
    count = len(codecs)
    if outs is None:
        outs = [torch.empty(c.pos_shape, dtype=torch.float64, device="cuda") for c in codecs]
    hs = _ptr_array([c._h.value for c in codecs])
    bs = _ptr_array([b.data_ptr() for b in bitstreams])
    nb = _ptr_array([b.numel() for b in bitstreams], ctypes.c_size_t)
    os_ = _ptr_array([o.data_ptr() for o in outs])
    sts = (ctypes.c_int * count)()
    st = lib.mesh_codec_decode_batch_ex(ctypes.cast(hs, _P), count, ctypes.cast(bs, _P),
                                        ctypes.cast(nb, _P), ctypes.cast(os_, _P),
                                        ctypes.cast(sts, _P),
                                        MC_BATCH_GROUPED if grouped else 0,
                                        _stream_ptr(stream))
    if not (allow_not_converged and st == 6):
        _check(st, "mesh_codec_decode_batch_ex")
    return outs


# ---------------------------------------------------------------- learned warm start
def _dptr(t, dtype=None, shape=None):
    torch = _torch()
    assert t.is_cuda and t.is_contiguous(), "CUDA contiguous tensor expected"
    if dtype is not None:
        assert t.dtype == dtype, f"{t.dtype} != {dtype}"
    if shape is not None:
        assert tuple(t.shape) == tuple(shape), f"{tuple(t.shape)} != {tuple(shape)}"
    del torch
    return ctypes.c_void_p(t.data_ptr())


class Mlp:
    """n_in -> n_hidden -> n_hidden -> n_out perceptron (ReLU), bfloat16
    weights, float32 accumulation, trained with Adam on a float32 master
    copy; see mesh_codec_mlp_create.  Rows are samples (float32 CUDA)."""

    def __init__(self, n_in, n_hidden=256, n_out=3, seed=0):
        self._lib = load_library()
        h = ctypes.c_void_p()
        _check(self._lib.mesh_codec_mlp_create(int(n_in), int(n_hidden), int(n_out),
                                               ctypes.c_uint64(seed & ((1 << 64) - 1)),
                                               ctypes.byref(h)), "mesh_codec_mlp_create")
        self._h = h
        self.n_in, self.n_hidden, self.n_out = int(n_in), int(n_hidden), int(n_out)
        self.count = int(self._lib.mesh_codec_mlp_param_count(h))

    def params(self, which=0, stream=None):
        """0: float32 master, 1: bfloat16 copy (as float32), 2: last gradient."""
        torch = _torch()
        out = torch.empty(self.count, dtype=torch.float32, device="cuda")
        _check(self._lib.mesh_codec_mlp_get_params(self._h, int(which), _dptr(out),
                                                   _stream_ptr(stream)),
               "mesh_codec_mlp_get_params")
        return out

    def set_params(self, flat, stream=None):
        torch = _torch()
        _check(self._lib.mesh_codec_mlp_set_params(self._h, _dptr(flat, torch.float32,
                                                                   (self.count,)),
                                                   _stream_ptr(stream)),
               "mesh_codec_mlp_set_params")

    def fit_normalizer(self, X, stream=None):
        """Standardise inputs by the column means / deviations of X."""
        torch = _torch()
        _check(self._lib.mesh_codec_mlp_fit_normalizer(
            self._h, _dptr(X, torch.float32, (X.shape[0], self.n_in)), X.shape[0],
            _stream_ptr(stream)), "mesh_codec_mlp_fit_normalizer")

    def normalizer(self, stream=None):
        torch = _torch()
        mu = torch.empty(self.n_in, dtype=torch.float32, device="cuda")
        inv = torch.empty(self.n_in, dtype=torch.float32, device="cuda")
        _check(self._lib.mesh_codec_mlp_get_normalizer(self._h, _dptr(mu), _dptr(inv),
                                                       _stream_ptr(stream)),
               "mesh_codec_mlp_get_normalizer")
        return mu, inv

    def set_check_mode(self, fp32_weights):
        _check(self._lib.mesh_codec_mlp_set_check_mode(self._h, int(bool(fp32_weights))),
               "mesh_codec_mlp_set_check_mode")

    def forward(self, X, out=None, stream=None):
        torch = _torch()
        N = X.shape[0]
        if out is None:
            out = torch.empty((N, self.n_out), dtype=torch.float32, device=X.device)
        _check(self._lib.mesh_codec_mlp_forward(self._h, _dptr(X, torch.float32, (N, self.n_in)),
                                                N, _dptr(out, torch.float32, (N, self.n_out)),
                                                _stream_ptr(stream)),
               "mesh_codec_mlp_forward")
        return out

    def infer(self, X, out=None, stream=None):
        """forward() with the hidden-to-hidden product on the tensor cores
        (TF32; mesh_codec_mlp_infer), for predictions over many rows."""
        torch = _torch()
        N = X.shape[0]
        if out is None:
            out = torch.empty((N, self.n_out), dtype=torch.float32, device=X.device)
        _check(self._lib.mesh_codec_mlp_infer(self._h, _dptr(X, torch.float32, (N, self.n_in)),
                                              N, _dptr(out, torch.float32, (N, self.n_out)),
                                              _stream_ptr(stream)),
               "mesh_codec_mlp_infer")
        return out

    def train_step(self, X, T, lr=1e-3, update=True, want_loss=True, stream=None):
        """One forward/backward pass (and an Adam step when update); returns
        the mean squared error (synchronising) or None."""
        torch = _torch()
        N = X.shape[0]
        loss = ctypes.c_double()
        _check(self._lib.mesh_codec_mlp_train_step(
            self._h, _dptr(X, torch.float32, (N, self.n_in)),
            _dptr(T, torch.float32, (N, self.n_out)), N, float(lr), int(bool(update)),
            ctypes.byref(loss) if want_loss else None, _stream_ptr(stream)),
            "mesh_codec_mlp_train_step")
        return loss.value if want_loss else None

    def close(self):
        if getattr(self, "_h", None):
            self._lib.mesh_codec_mlp_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


WARM_ANCHORS = 3
WARM_FEATURES = 16


def farthest_anchors(xyz, n_anchors, start=0, stream=None):
    """n_anchors vertices spread over the pose xyz (CUDA float64 [n, 3]) by
    greedy farthest-point selection from vertex `start`: CUDA int32
    [n_anchors], ascending (mesh_codec_farthest_anchors)."""
    torch = _torch()
    n = xyz.shape[0]
    out = torch.empty(int(n_anchors), dtype=torch.int32, device=xyz.device)
    _check(load_library().mesh_codec_farthest_anchors(
        n, int(n_anchors), _dptr(xyz, torch.float64, (n, 3)), int(start), _dptr(out),
        _stream_ptr(stream)), "mesh_codec_farthest_anchors")
    return out


def nearest_anchors(rest, anchors, stream=None):
    """rest: CUDA float64 [n, 3]; anchors: CUDA int32 [n_c] ->
    (int32 [n, 3] indices into anchors, float32 [n, 3] distances)."""
    torch = _torch()
    n, n_c = rest.shape[0], anchors.shape[0]
    idx = torch.empty((n, WARM_ANCHORS), dtype=torch.int32, device=rest.device)
    dist = torch.empty((n, WARM_ANCHORS), dtype=torch.float32, device=rest.device)
    _check(load_library().mesh_codec_nearest_anchor(
        n, n_c, _dptr(rest, torch.float64, (n, 3)), _dptr(anchors, torch.int32, (n_c,)),
        _dptr(idx), _dptr(dist), _stream_ptr(stream)), "mesh_codec_nearest_anchor")
    return idx, dist


def warm_features(x_last, a_cur, anchors, nearest, dist, delta_cur, delta_prev, dscale=1.0,
                  x_cur=None, stream=None):
    """Features (float32 [F*n, 16]) and, with x_cur, targets (float32
    [F*n, 3]); see mesh_codec_warm_features for the layouts."""
    torch = _torch()
    n = x_last.shape[0]
    n_c, F = a_cur.shape[1], a_cur.shape[2]
    a_cur = a_cur.contiguous()
    feat = torch.empty((n * F, WARM_FEATURES), dtype=torch.float32, device=x_last.device)
    tgt = None
    if x_cur is not None:
        tgt = torch.empty((n * F, 3), dtype=torch.float32, device=x_last.device)
    f64 = torch.float64
    _check(load_library().mesh_codec_warm_features(
        n, F, n_c, _dptr(x_last, f64, (n, 3)), _dptr(a_cur, f64, (3, n_c, F)),
        _dptr(anchors, torch.int32, (n_c,)), _dptr(nearest, torch.int32, (n, WARM_ANCHORS)),
        _dptr(dist, torch.float32, (n, WARM_ANCHORS)), _dptr(delta_cur, f64, (n, 3 * F)),
        _dptr(delta_prev, f64, (n, 3 * F)), float(dscale),
        None if x_cur is None else _dptr(x_cur, f64, (F, n, 3)), _dptr(feat),
        None if tgt is None else _dptr(tgt), _stream_ptr(stream)), "mesh_codec_warm_features")
    return feat, tgt


def warm_compose(x_last, F, pred=None, stream=None):
    """x0 [F, n, 3] float64 = x_last (+ pred reshaped to [F, n, 3])."""
    torch = _torch()
    n = x_last.shape[0]
    x0 = torch.empty((F, n, 3), dtype=torch.float64, device=x_last.device)
    _check(load_library().mesh_codec_warm_compose(
        n, F, _dptr(x_last, torch.float64, (n, 3)),
        None if pred is None else _dptr(pred, torch.float32, (n * F, 3)), _dptr(x0),
        _stream_ptr(stream)), "mesh_codec_warm_compose")
    return x0


def sample_rows(X, seed, count, stream=None):
    """Rows splitmix64(seed)_i mod N of a float32 [N, w] CUDA tensor."""
    torch = _torch()
    N, w = X.shape
    out = torch.empty((int(count), w), dtype=torch.float32, device=X.device)
    _check(load_library().mesh_codec_sample_rows(_dptr(X, torch.float32), w, N,
                                                 ctypes.c_uint64(seed & ((1 << 64) - 1)),
                                                 int(count), _dptr(out), _stream_ptr(stream)),
           "mesh_codec_sample_rows")
    return out


def basis_features(U_prev, U_cur=None, stream=None):
    """U [3, F, k] float64 -> (features float32 [3F, k+1], target [3F, k] or None)."""
    torch = _torch()
    _, F, k = U_prev.shape
    feat = torch.empty((3 * F, k + 1), dtype=torch.float32, device=U_prev.device)
    tgt = None if U_cur is None else torch.empty((3 * F, k), dtype=torch.float32,
                                                 device=U_prev.device)
    _check(load_library().mesh_codec_basis_features(
        F, k, _dptr(U_prev, torch.float64, (3, F, k)),
        None if U_cur is None else _dptr(U_cur, torch.float64, (3, F, k)), _dptr(feat),
        None if tgt is None else _dptr(tgt), _stream_ptr(stream)), "mesh_codec_basis_features")
    return feat, tgt


def basis_compose(U_prev, pred=None, stream=None):
    torch = _torch()
    _, F, k = U_prev.shape
    q0 = torch.empty((3, F, k), dtype=torch.float64, device=U_prev.device)
    _check(load_library().mesh_codec_basis_compose(
        F, k, _dptr(U_prev, torch.float64, (3, F, k)),
        None if pred is None else _dptr(pred, torch.float32, (3 * F, k)), _dptr(q0),
        _stream_ptr(stream)), "mesh_codec_basis_compose")
    return q0


def rates(n_blocks=1, **kw):
    """Eq. 13's bits per vertex and frame for a stream of the given
    parameters (see mesh_codec_rates): {q, q_a, q_d, q_s, stream}."""
    p = default_params()
    for key, val in kw.items():
        if not hasattr(p, key):
            raise TypeError(f"unknown parameter {key}")
        setattr(p, key, val)
    out = (ctypes.c_double * 5)()
    _check(load_library().mesh_codec_rates(ctypes.byref(p), int(n_blocks),
                                           ctypes.cast(out, ctypes.c_void_p)), "mesh_codec_rates")
    return dict(zip(("q", "q_a", "q_d", "q_s", "stream"), list(out)))
