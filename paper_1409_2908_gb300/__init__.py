"""GB300-native recursive fast matrix multiplication (Benson & Ballard,
"A Framework for Practical Parallel Fast Matrix Multiplication").

Thin Python binding over the C ABI of libfmm.so (include/fmm.h): it only
marshals arguments.  Every step of a product runs in the library's CUDA
kernels; PyTorch supplies device memory and streams.  There is no CPU path.
"""
import ctypes
import os

from . import _lib

FMM_OK = 0
FMM_ERR_ARG = -1
FMM_ERR_INVALID_ALGORITHM = -2
FMM_ERR_UNSUPPORTED = -3
FMM_ERR_NO_MEMORY = -4
FMM_ERR_CUDA = -5
FMM_ERR_TIMEOUT = -6

FMM_PREC_FP64 = 0
FMM_PREC_OZAKI_BF16 = 3
FMM_PREC_TF32 = 2
FMM_PREC_FP32 = 1
PRECISIONS = {"fp64": FMM_PREC_FP64, "ozaki_bf16": FMM_PREC_OZAKI_BF16, "tf32": FMM_PREC_TF32,
              "fp32": FMM_PREC_FP32}
FLAG_FUSED_ST = 1
FLAG_FUSED_W = 2
FLAG_LEVELWISE = 4
FLAG_LEAF_EMULATION = 8
FLAG_STREAMING = 16
FLAG_PAIRWISE = 32
FLAG_TC_FUSED_S = 64
FLAGS_DEFAULT = FLAG_FUSED_ST | FLAG_FUSED_W

TILES = {"auto": 0, "128x128": 1, "96x96": 2, "64x64": 3, "32x32": 4, "128x64": 5, "64x128": 6}

ALGORITHM_DIR = os.path.join(os.path.dirname(os.path.abspath(__file__)), "algorithms")


class FmmError(RuntimeError):
    def __init__(self, status, what=""):
        self.status = status
        msg = _lib.lib().fmm_status_string(status).decode()
        super().__init__(f"{what}: {msg} ({status})" if what else f"{msg} ({status})")


def _check(status, what):
    if status != FMM_OK:
        raise FmmError(status, what)


def algorithm_path(name):
    """Path of a shipped algorithm file, e.g. 'strassen_222_7'."""
    p = name if os.path.isabs(name) else os.path.join(ALGORITHM_DIR, name)
    if not p.endswith(".fmm"):
        p += ".fmm"
    return p


def _stream_handle(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if isinstance(stream, int):
        return ctypes.c_void_p(stream)
    return ctypes.c_void_p(stream.cuda_stream)


def _mat(t, name):
    """(pointer, leading dimension, rows, cols) of a row-major FP64 matrix;
    a torch CUDA tensor or anything exposing a data pointer and strides."""
    if t.dim() != 2 or t.dtype.is_floating_point is False:
        raise ValueError(f"{name} must be a 2-D floating tensor")
    import torch
    if t.dtype != torch.float64:
        raise ValueError(f"{name} must be float64")
    if t.stride(1) != 1:
        raise ValueError(f"{name} must have unit column stride")
    return ctypes.c_void_p(t.data_ptr()), max(t.stride(0), t.shape[1]), t.shape[0], t.shape[1]


def algorithm_factors(name):
    """(M, K, N, U, V, W) of a shipped algorithm file: U is MK x R, V is KN x R,
    W is MN x R (rows in row-order vec of A, B, C; Section 2.2.2).  Entries
    may be written as fractions a/b."""
    import numpy as np
    from fractions import Fraction
    with open(algorithm_path(name)) as fh:
        toks = [ln.split("#", 1)[0].split() for ln in fh]
    toks = [t for t in toks if t]
    M, K, N, R = (int(x) for x in toks[0])
    mats, cur = {}, None
    for t in toks[1:]:
        if len(t) == 1 and t[0] in ("U", "V", "W"):
            cur = mats.setdefault(t[0], [])
        else:
            cur.append([float(Fraction(x)) for x in t])
    U, V, W = (np.array(mats[k], dtype=np.float64).reshape(-1, R) for k in ("U", "V", "W"))
    return M, K, N, U, V, W


class Plan:
    """A fast-multiplication plan: base case [[U,V,W]] unrolled over `levels`
    recursive steps (fmm_plan_create / fmm_plan_load)."""

    def __init__(self, algorithm=None, levels=1, flags=FLAGS_DEFAULT, tile="auto", factors=None,
                 precision="fp64", moduli=None):
        L = _lib.lib()
        prec = PRECISIONS[precision]
        h = ctypes.c_void_p()
        if factors is not None:
            import numpy as np
            M, K, N, U, V, W = factors
            U = np.ascontiguousarray(U, dtype=np.float64)
            V = np.ascontiguousarray(V, dtype=np.float64)
            W = np.ascontiguousarray(W, dtype=np.float64)
            R = U.shape[1]
            st = L.fmm_plan_create(ctypes.byref(h), M, K, N, R, U.ctypes.data, V.ctypes.data,
                                   W.ctypes.data, levels, prec, flags)
        else:
            st = L.fmm_plan_load(ctypes.byref(h), algorithm_path(algorithm).encode(), levels,
                                 prec, flags)
        _check(st, "plan")
        self._h = h
        self.levels = levels
        self.flags = flags
        self.name = algorithm if factors is None else "custom"
        self.precision = precision
        self.moduli = moduli if precision == "ozaki_bf16" else None
        self.tile = tile
        if tile != "auto":
            self.set_tile(tile)
        if moduli is not None:
            _check(L.fmm_plan_set_moduli(self._h, int(moduli)), "set_moduli")

    def prepare(self):
        """Upload the plan and set up its kernels now (before graph capture)."""
        _check(_lib.lib().fmm_plan_prepare(self._h), "prepare")

    def set_tile(self, tile):
        _check(_lib.lib().fmm_plan_set_tile(self._h, TILES[tile]), "set_tile")

    @property
    def handle(self):
        return self._h

    @property
    def dims(self):
        """(M, K, N) of the base case."""
        inf = self.info()
        return inf["M"], inf["K"], inf["N"]

    @property
    def rank(self):
        """R, the base case's number of products."""
        return self.info()["R"]

    def info(self):
        inf = _lib.PlanInfo()
        _check(_lib.lib().fmm_plan_info(self._h, ctypes.byref(inf)), "info")
        return {f: getattr(inf, f) for f, _ in inf._fields_}

    def leaf_terms(self, which):
        """(ptr, row, col, coef) numpy arrays of the unrolled lists of
        operand `which` (0: A/U, 1: B/V, 2: C/W)."""
        import numpy as np
        inf = self.info()
        n = inf[("nnz_a_terms", "nnz_b_terms", "nnz_c_terms")[which]]
        ptr = np.zeros(inf["leaves"] + 1, np.int64)
        row = np.zeros(n, np.int32)
        col = np.zeros(n, np.int32)
        coef = np.zeros(n, np.float64)
        _check(_lib.lib().fmm_plan_leaf_terms(self._h, which, ptr.ctypes.data, row.ctypes.data,
                                              col.ctypes.data, coef.ctypes.data, n), "leaf_terms")
        return ptr, row, col, coef

    def workspace_size(self, m, k, n):
        b = ctypes.c_size_t()
        _check(_lib.lib().fmm_workspace_size(self._h, m, k, n, ctypes.byref(b)), "workspace_size")
        return b.value

    def host_workspace_size(self, m, k, n):
        b = ctypes.c_size_t()
        _check(_lib.lib().fmm_host_workspace_size(self._h, m, k, n, ctypes.byref(b)),
               "host_workspace_size")
        return b.value

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            _lib.lib().fmm_plan_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _alloc_ws(nbytes, device):
    import torch
    if nbytes == 0:
        return None
    return torch.empty(nbytes, dtype=torch.uint8, device=device)


def gemm(plan, A, B, C=None, workspace=None, stream=None):
    """C = A B with the plan's fast algorithm (fmm_gemm).  A, B, C: CUDA
    float64 tensors, row-major.  Returns C."""
    import torch
    pa, lda, m, k = _mat(A, "A")
    pb, ldb, k2, n = _mat(B, "B")
    if k2 != k:
        raise ValueError("inner dimensions differ")
    if C is None:
        C = torch.empty((m, n), dtype=torch.float64, device=A.device)
    pc, ldc, m2, n2 = _mat(C, "C")
    if (m2, n2) != (m, n):
        raise ValueError("C has the wrong shape")
    need = plan.workspace_size(m, k, n)
    if workspace is None:
        workspace = _alloc_ws(need, A.device)
    wptr = ctypes.c_void_p(workspace.data_ptr()) if workspace is not None else ctypes.c_void_p()
    wbytes = workspace.numel() * workspace.element_size() if workspace is not None else 0
    st = _lib.lib().fmm_gemm(plan.handle, pa, lda, pb, ldb, pc, ldc, m, k, n, wptr, wbytes,
                             _stream_handle(stream))
    _check(st, "fmm_gemm")
    return C


def gemm_batched(plan, As, Bs, Cs=None, workspace=None, stream=None):
    """C_b = A_b B_b for equally shaped CUDA float64 tensors, all leaves of all
    products in one grouped launch (fmm_gemm_batched).  Returns the C list."""
    import torch
    count = len(As)
    if count != len(Bs) or count == 0:
        raise ValueError("need equally many A and B")
    mats = [_mat(a, "A") for a in As]
    matsb = [_mat(b, "B") for b in Bs]
    m, k = mats[0][2], mats[0][3]
    n = matsb[0][3]
    if Cs is None:
        Cs = [torch.empty((m, n), dtype=torch.float64, device=As[0].device) for _ in range(count)]
    matsc = [_mat(c, "C") for c in Cs]
    lda, ldb, ldc = mats[0][1], matsb[0][1], matsc[0][1]
    if any(x[1] != lda or x[2:] != (m, k) for x in mats) or any(x[1] != ldb or x[2:] != (k, n) for x in matsb) \
            or any(x[1] != ldc or x[2:] != (m, n) for x in matsc):
        raise ValueError("batched operands must share shape and leading dimension")
    arr = ctypes.c_void_p * count
    pa = arr(*[x[0].value for x in mats])
    pb = arr(*[x[0].value for x in matsb])
    pc = arr(*[x[0].value for x in matsc])
    need = ctypes.c_size_t()
    _check(_lib.lib().fmm_workspace_size_batched(plan.handle, count, m, k, n, ctypes.byref(need)),
           "workspace_size_batched")
    if workspace is None:
        workspace = torch.empty(need.value, dtype=torch.uint8, device=As[0].device)
    st = _lib.lib().fmm_gemm_batched(plan.handle, count, pa, lda, pb, ldb, pc, ldc, m, k, n,
                                     ctypes.c_void_p(workspace.data_ptr()),
                                     workspace.numel() * workspace.element_size(),
                                     _stream_handle(stream))
    _check(st, "fmm_gemm_batched")
    return Cs


def gemm_grouped(plans, As, Bs, Cs=None, workspaces=None, stream=None):
    """C_i = A_i B_i for products of any shapes, each with its own plan, issued
    together (fmm_gemm_grouped): the emulated products' residue GEMMs share
    grouped tensor-core launches.  Returns the C list."""
    import torch
    count = len(plans)
    if count == 0 or len(As) != count or len(Bs) != count:
        raise ValueError("need one A and one B per plan")
    ma = [_mat(a, "A") for a in As]
    mb = [_mat(b, "B") for b in Bs]
    if any(x[3] != y[2] for x, y in zip(ma, mb)):
        raise ValueError("inner dimensions differ")
    if Cs is None:
        Cs = [torch.empty((x[2], y[3]), dtype=torch.float64, device=a.device) for x, y, a in zip(ma, mb, As)]
    mc = [_mat(c, "C") for c in Cs]
    if workspaces is None:
        workspaces = [_alloc_ws(p.workspace_size(x[2], x[3], y[3]), a.device) for p, x, y, a in zip(plans, ma, mb, As)]
    P = ctypes.c_void_p * count
    I64 = ctypes.c_int64 * count
    SZ = ctypes.c_size_t * count
    ws_ptr = P(*[w.data_ptr() if w is not None else None for w in workspaces])
    ws_b = SZ(*[w.numel() * w.element_size() if w is not None else 0 for w in workspaces])
    st = _lib.lib().fmm_gemm_grouped(
        count, P(*[p.handle.value for p in plans]), P(*[x[0].value for x in ma]), I64(*[x[1] for x in ma]),
        P(*[x[0].value for x in mb]), I64(*[x[1] for x in mb]), P(*[x[0].value for x in mc]),
        I64(*[x[1] for x in mc]), I64(*[x[2] for x in ma]), I64(*[x[3] for x in ma]), I64(*[x[3] for x in mb]),
        ws_ptr, ws_b, _stream_handle(stream))
    _check(st, "fmm_gemm_grouped")
    return Cs


def classical_gemm(A, B, C=None, stream=None):
    """C = A B with the library's classical FP64 GEMM (fmm_classical_gemm)."""
    import torch
    pa, lda, m, k = _mat(A, "A")
    pb, ldb, k2, n = _mat(B, "B")
    if k2 != k:
        raise ValueError("inner dimensions differ")
    if C is None:
        C = torch.empty((m, n), dtype=torch.float64, device=A.device)
    pc, ldc, _, _ = _mat(C, "C")
    st = _lib.lib().fmm_classical_gemm(pa, lda, pb, ldb, pc, ldc, m, k, n, _stream_handle(stream))
    _check(st, "fmm_classical_gemm")
    return C


def gemm_host(plan, A, B, C, dev_ws, stream=None):
    """End-to-end product of HOST matrices (fmm_gemm_host): A, B, C are CPU
    float64 tensors (ideally pinned), dev_ws a CUDA byte tensor of
    host_workspace_size() bytes.  plan=None uses the classical GEMM."""
    pa, lda, m, k = _mat(A, "A")
    pb, ldb, k2, n = _mat(B, "B")
    pc, ldc, _, _ = _mat(C, "C")
    h = plan.handle if plan is not None else ctypes.c_void_p()
    st = _lib.lib().fmm_gemm_host(h, pa, lda, pb, ldb, pc, ldc, m, k, n,
                                  ctypes.c_void_p(dev_ws.data_ptr()),
                                  dev_ws.numel() * dev_ws.element_size(), _stream_handle(stream))
    _check(st, "fmm_gemm_host")
    return C


def set_host_pipeline(bands=0, gemm_bands=0):
    """Overlap depth of later gemm_host calls on this thread
    (fmm_set_host_pipeline): C copied out in `bands` row bands, residue
    products made in `gemm_bands` row bands; 0 = chosen from the sizes."""
    _check(_lib.lib().fmm_set_host_pipeline(int(bands), int(gemm_bands)), "set_host_pipeline")


def host_workspace_size(plan, m, k, n):
    b = ctypes.c_size_t()
    h = plan.handle if plan is not None else ctypes.c_void_p()
    _check(_lib.lib().fmm_host_workspace_size(h, m, k, n, ctypes.byref(b)), "host_workspace_size")
    return b.value


def last_launch_count():
    """Kernel launches enqueued by the last gemm / classical_gemm call on this thread."""
    return _lib.lib().fmm_last_launch_count()


def check_device_error():
    """Raise FmmError(FMM_ERR_TIMEOUT) if a bounded device wait gave up."""
    _check(_lib.lib().fmm_check_device_error(), "device")


def set_wait_limit(ns):
    """Time limit (ns) of the tensor-core kernels' bounded waits (fmm_set_wait_limit)."""
    _check(_lib.lib().fmm_set_wait_limit(int(ns)), "set_wait_limit")


def selftest_wait_timeout(kernel, ns, stream=None):
    """Status of fmm_selftest_wait_timeout: FMM_ERR_TIMEOUT when the dry
    kernel's wait ran out as it should (kernel 0: residue GEMM, 1: TF32)."""
    return _lib.lib().fmm_selftest_wait_timeout(int(kernel), int(ns), _stream_handle(stream))


def timing_enable(on=True):
    """Record CUDA events around each call's leaf-product launch (this thread)."""
    _check(_lib.lib().fmm_timing_enable(1 if on else 0), "timing_enable")


def timing_leaf_ms():
    """(summed milliseconds, calls) of the recorded leaf launches; clears them."""
    ms = ctypes.c_double()
    cnt = ctypes.c_int()
    _check(_lib.lib().fmm_timing_leaf_ms(ctypes.byref(ms), ctypes.byref(cnt)), "timing_leaf_ms")
    return ms.value, cnt.value


def library_path():
    return _lib.path()
