"""Thin Python front end of the C ABI: operator descriptors holding torch device tensors and a
``Solver`` whose methods map one-to-one onto sgks_create / sgks_reset / sgks_step /
sgks_solve / sgks_destroy.  Every step of the method runs in the CUDA library; this module
only builds the descriptor structs and passes device pointers and the current stream.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass
from typing import Optional

import torch

from . import _lib as L


# Precision forms (the precision field of sgks_options):
#   "fp64"       everything FP64;
#   "fp32"       FP32 basis, operator values and b; the sketch inputs, x, e and the gradient in
#                compensated float-float arithmetic on the FP32 units; FP64 small phase
#                ("fp32x" is the same form);
#   "fp32plain"  FP32 arithmetic with FP32 accumulation in the operator passes (drifts from the
#                FP64 iterates; kept for comparison);
#   "ff"         batches only: the basis and every vector in float-float, FP64-class results.
PRECISIONS = {"fp64": L.SGKS_PREC_FP64, "fp32": L.SGKS_PREC_FP32, "fp32x": L.SGKS_PREC_FP32X,
              "fp32plain": L.SGKS_PREC_FP32_PLAIN, "ff": L.SGKS_PREC_FF}


def io_dtype(precision):
    """Element type of b, x_true and x at the interface for a precision form."""
    if precision not in PRECISIONS:
        raise ValueError(f"unknown precision {precision!r}")
    return torch.float32 if precision in ("fp32", "fp32x", "fp32plain") else torch.float64


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _need_cuda(t, name):
    if t is not None and not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t is not None and not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


@dataclass
class CSR:
    """A (m x n) as CSR: row_ptr[m+1], col[nnz] int32; val[nnz] float32/float64 (device)."""
    row_ptr: torch.Tensor
    col: torch.Tensor
    val: torch.Tensor
    m: int
    n: int
    t_row_ptr: Optional[torch.Tensor] = None
    t_col: Optional[torch.Tensor] = None
    t_val: Optional[torch.Tensor] = None

    def desc(self):
        for nm in ("row_ptr", "col", "val", "t_row_ptr", "t_col", "t_val"):
            _need_cuda(getattr(self, nm), nm)
        d = L.sgks_op()
        d.kind, d.m, d.n = L.SGKS_OP_CSR, self.m, self.n
        d.val_dtype = L.SGKS_F64 if self.val.dtype == torch.float64 else L.SGKS_F32
        d.nnz = int(self.col.numel())
        d.row_ptr, d.col, d.val = _ptr(self.row_ptr), _ptr(self.col), _ptr(self.val)
        d.t_row_ptr, d.t_col, d.t_val = _ptr(self.t_row_ptr), _ptr(self.t_col), _ptr(self.t_val)
        return d

    def transposed(self, stream=None):
        """Build the column storage of A on the device (sgks_csr_transpose) and keep it."""
        lib = L.load()
        dev = self.col.device
        self.t_row_ptr = torch.empty(self.n + 1, dtype=torch.int32, device=dev)
        self.t_col = torch.empty_like(self.col)
        self.t_val = torch.empty_like(self.val)
        vd = L.SGKS_F64 if self.val.dtype == torch.float64 else L.SGKS_F32
        st = torch.cuda.current_stream(dev).cuda_stream if stream is None else stream
        L.check(lib.sgks_csr_transpose(self.m, self.n, int(self.col.numel()), _ptr(self.row_ptr), _ptr(self.col),
                                       _ptr(self.val), vd, _ptr(self.t_row_ptr), _ptr(self.t_col),
                                       _ptr(self.t_val), C.c_void_p(st)))
        return self


@dataclass
class Dense:
    """A (m x n) dense, row-major, float32/float64 (device)."""
    mat: torch.Tensor

    def desc(self):
        _need_cuda(self.mat, "mat")
        d = L.sgks_op()
        d.kind = L.SGKS_OP_DENSE
        d.m, d.n = self.mat.shape
        d.ld = self.mat.shape[1]
        d.val_dtype = L.SGKS_F64 if self.mat.dtype == torch.float64 else L.SGKS_F32
        d.dense = _ptr(self.mat)
        return d


@dataclass
class Conv2D:
    """2D convolution of an (ny, nx) image with the odd-sized psf (kh, kw), zero boundary."""
    psf: torch.Tensor
    nx: int
    ny: int

    def desc(self):
        _need_cuda(self.psf, "psf")
        d = L.sgks_op()
        d.kind = L.SGKS_OP_CONV2D
        d.m = d.n = self.nx * self.ny
        d.nx, d.ny = self.nx, self.ny
        d.kh, d.kw = self.psf.shape
        d.val_dtype = L.SGKS_F64 if self.psf.dtype == torch.float64 else L.SGKS_F32
        d.psf = _ptr(self.psf)
        return d


_REG = {"fd1": L.SGKS_REG_FD1, "grad2d": L.SGKS_REG_GRAD2D, "laplace2d": L.SGKS_REG_LAPLACE2D,
        "spacetime": L.SGKS_REG_SPACETIME}


@dataclass
class Reg:
    """Matrix-free finite-difference L: kind in fd1 / grad2d / laplace2d / spacetime."""
    kind: str
    nx: int
    ny: int = 1
    nt: int = 1

    def desc(self):
        r = L.sgks_reg()
        r.kind, r.nx, r.ny, r.nt = _REG[self.kind], self.nx, self.ny, self.nt
        return r


class Solver:
    """sGKS solver (Algorithm 2; method="gks": GKS, Algorithm 1) on the current CUDA device and stream.

    A: CSR | Dense | Conv2D; L: Reg; b: device tensor (float64 for precision="fp64", float32
    for "fp32"); lam > 0; sketch_rows = s.  Tensors passed here must outlive the solver.
    """

    def __init__(self, A, reg: Reg, b: torch.Tensor, lam: float, sketch_rows: int, seed: int = 0, *,
                 max_iters: int = 100, ell: int = 3, n_refine: int = 0, precision: str = "fp64",
                 sketch: str = "sparse_sign", zeta: int = 8, cgs_passes: int = 2,
                 gauss_SA: Optional[torch.Tensor] = None, gauss_SL: Optional[torch.Tensor] = None,
                 x_true: Optional[torch.Tensor] = None, stream=None, flags: int = 0, record: bool = False,
                 method: str = "sgks", srtt=None):
        self._lib = L.load()
        self.precision = precision
        self.dtype = io_dtype(precision)
        for nm, t in (("b", b), ("x_true", x_true)):
            _need_cuda(t, nm)
            if t is not None and t.dtype != self.dtype:
                raise ValueError(f"{nm} must be {self.dtype} for precision={precision}")
        for nm, t in (("gauss_SA", gauss_SA), ("gauss_SL", gauss_SL)):
            _need_cuda(t, nm)
            if t is not None and t.dtype != torch.float64:
                raise ValueError(f"{nm} must be float64")
        self._keep = [A, b, x_true, gauss_SA, gauss_SL]
        self.A, self.reg = A, reg
        self.n = A.desc().n
        self.m = A.desc().m
        self.lam = float(lam)
        self.max_iters = max_iters
        o = L.sgks_options()
        o.max_iters, o.ell, o.n_refine, o.zeta, o.cgs_passes = max_iters, ell, n_refine, zeta, cgs_passes
        o.precision = PRECISIONS[precision]
        o.sketch_kind = {"gaussian": L.SGKS_SKETCH_GAUSSIAN, "srtt": L.SGKS_SKETCH_SRTT}.get(
            sketch, L.SGKS_SKETCH_SPARSE_SIGN)
        o.gauss_SA, o.gauss_SL, o.x_true = _ptr(gauss_SA), _ptr(gauss_SL), _ptr(x_true)
        if sketch == "srtt":
            if srtt is None or len(srtt) != 4:
                raise ValueError("sketch='srtt' needs srtt=(signs_A int8, rows_A int32, signs_L int8, rows_L int32)")
            for t, nm in zip(srtt, ("signs_A", "rows_A", "signs_L", "rows_L")):
                _need_cuda(t, nm)
            self._keep.append(srtt)
            o.srtt_signs_A, o.srtt_rows_A, o.srtt_signs_L, o.srtt_rows_L = [_ptr(t) for t in srtt]
        if method not in ("sgks", "gks"):
            raise ValueError("method is 'sgks' (Algorithm 2) or 'gks' (Algorithm 1)")
        o.flags = int(flags) | (L.SGKS_FLAG_RECORD if record else 0) | (L.SGKS_FLAG_GKS if method == "gks" else 0)
        self._stream = torch.cuda.current_stream(b.device).cuda_stream if stream is None else stream
        self.device = b.device
        h = C.c_void_p()
        self._adesc, self._rdesc = A.desc(), reg.desc()
        rc = self._lib.sgks_create(C.byref(h), C.byref(self._adesc), C.byref(self._rdesc), _ptr(b), float(lam),
                                   int(sketch_rows), int(seed), C.byref(o), C.c_void_p(self._stream))
        L.check(rc, None)
        self._h = h

    # -- Algorithm 2 -----------------------------------------------------------------
    def reset(self, b: torch.Tensor):
        _need_cuda(b, "b")
        self._keep[1] = b
        L.check(self._lib.sgks_reset(self._h, _ptr(b)), self._h)

    def step(self):
        L.check(self._lib.sgks_step(self._h), self._h)

    def solve(self, iters: int, tol: float = 0.0, x_out: Optional[torch.Tensor] = None, history: bool = False):
        rep = L.sgks_report()
        rc_arr = (C.c_double * max(iters, 1))() if history else None
        rre_arr = (C.c_double * max(iters, 1))() if history else None
        if history:
            rep.rc = C.cast(rc_arr, C.POINTER(C.c_double))
            rep.rre = C.cast(rre_arr, C.POINTER(C.c_double))
        if x_out is not None:
            _need_cuda(x_out, "x_out")
        L.check(self._lib.sgks_solve(self._h, int(iters), float(tol), _ptr(x_out), C.byref(rep)), self._h)
        out = dict(iters_done=rep.iters_done, status=rep.status, d=rep.subspace_dim, rc_last=rep.rc_last,
                   rre_last=rep.rre_last, rre0=rep.rre0)
        if history:
            out["rc"] = list(rc_arr[:rep.iters_done])
            out["rre"] = list(rre_arr[:rep.iters_done])
        return out

    def status(self):
        c = C.c_int32()
        L.check(self._lib.sgks_status(self._h, C.byref(c)), self._h)
        return c.value

    def info(self):
        a = (C.c_int64 * 3)()
        L.check(self._lib.sgks_get_info(self._h, a), self._h)
        return dict(d=a[0], iter=a[1], status=a[2])

    # -- inspection -------------------------------------------------------------------
    def buffer(self, which: int, count: int, dtype=torch.float64):
        out = torch.empty(count, dtype=dtype, device=self.device)
        n = C.c_size_t()
        L.check(self._lib.sgks_get_buffer(self._h, which, _ptr(out), out.numel() * out.element_size(),
                                          C.byref(n)), self._h)
        return out[: n.value // out.element_size()]

    def x(self):
        """Current iterate x_k.  The compensated FP32 form keeps x as float-float pairs, which are
        summed in float64 here."""
        if self.dtype == torch.float32:
            v = self.buffer(L.SGKS_BUF_X, 2 * self.n, torch.float32)
            if v.numel() == 2 * self.n:
                v = v.view(self.n, 2).double()
                return v[:, 0] + v[:, 1]
            return v
        return self.buffer(L.SGKS_BUF_X, self.n, self.dtype)

    def apply(self, which: int, x: torch.Tensor, out: torch.Tensor):
        L.check(self._lib.sgks_apply(self._h, which, _ptr(x), _ptr(out)), self._h)
        return out

    def profile(self, iters: int, graph: bool = False):
        """Per-kernel CUDA-event timing of `iters` iterations: eager launches with a synchronised
        event pair around each (sgks_profile_steps), or, with graph=True, event pairs recorded as
        nodes of one captured graph (sgks_profile_graph), kernels back to back as in solve()."""
        n = L.SGKS_PROFILE_CLASSES
        ms, cnt, ds = (C.c_double * n)(), (C.c_int64 * n)(), (C.c_double * n)()
        fn = self._lib.sgks_profile_graph if graph else self._lib.sgks_profile_steps
        L.check(fn(self._h, int(iters), ms, cnt, ds), self._h)
        return {L.PROFILE_CLASS_NAMES[i]: dict(ms=ms[i], launches=cnt[i], dsum=ds[i]) for i in range(n)}

    def time_class(self, name: str, reps: int = 100) -> float:
        """Microseconds per launch of one streaming kernel class ("gradient_append",
        "sketch_column", "combine_refine", "gradient_refine") in the current state, from `reps`
        back-to-back launches in one CUDA graph (sgks_time_class); the iteration state is unchanged."""
        us = C.c_double()
        cls = L.PROFILE_CLASS_NAMES.index(name)
        L.check(self._lib.sgks_time_class(self._h, cls, int(reps), C.byref(us)), self._h)
        return us.value

    def set_lambda(self, lam: float):
        """Change lambda; the basis is discarded, so call reset(b) before the next step/solve."""
        L.check(self._lib.sgks_set_lambda(self._h, float(lam)), self._h)
        self.lam = float(lam)

    def backward(self, xbar: torch.Tensor):
        """(dl/db, dl/dlambda) for xbar = dl/dx_K of the iterations since the last setup
        (sgks_backward; the solver must have been created with record=True).  The sweep runs
        back through any refinement steps; repeated calls with the same K and lambda replay a
        captured CUDA graph of it."""
        _need_cuda(xbar, "xbar")
        if xbar.dtype != self.dtype or xbar.numel() != self.n:
            raise ValueError(f"xbar must hold {self.n} values of {self.dtype}")
        bbar = torch.empty(self.m, dtype=self.dtype, device=self.device)
        lb = C.c_double()
        L.check(self._lib.sgks_backward(self._h, _ptr(xbar), _ptr(bbar), C.byref(lb)), self._h)
        return bbar, lb.value

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sgks_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """Many independent sGKS problems in one handle (sgks_batch_*).

    instances: list of dicts with keys A (CSR | Dense | Conv2D), reg (Reg), b (device tensor of
    the solver precision), lam (> 0) and optionally x_true.  Instances whose A and reg describe
    the same device arrays and shape share the operator and run as interleaved groups; the
    others (ragged sizes) form groups of their own.  sketch_rows, seed and the options are shared
    and have the meaning they have for ``Solver``.  Tensors must outlive the batch.
    """

    def __init__(self, instances, sketch_rows: int, seed: int = 0, *, max_iters: int = 100, ell: int = 3,
                 n_refine: int = 0, precision: str = "fp64", zeta: int = 8, cgs_passes: int = 2, stream=None,
                 autotune: bool = False, tiles: bool = True):
        self._lib = L.load()
        self.precision = precision
        self.dtype = io_dtype(precision)
        k = len(instances)
        if k < 1:
            raise ValueError("a batch needs at least one instance")
        has_xt = all(inst.get("x_true") is not None for inst in instances)
        for inst in instances:
            for nm in ("b", "x_true"):
                t = inst.get(nm)
                _need_cuda(t, nm)
                if t is not None and t.dtype != self.dtype:
                    raise ValueError(f"{nm} must be {self.dtype} for precision={precision}")
        self._keep = [[inst["A"], inst["b"], inst.get("x_true")] for inst in instances]
        self.count = k
        self.n = [inst["A"].desc().n for inst in instances]
        self._adesc = (L.sgks_op * k)(*[inst["A"].desc() for inst in instances])
        self._rdesc = (L.sgks_reg * k)(*[inst["reg"].desc() for inst in instances])
        self._b = (C.c_void_p * k)(*[inst["b"].data_ptr() for inst in instances])
        self._lam = (C.c_double * k)(*[float(inst["lam"]) for inst in instances])
        self._xt = (C.c_void_p * k)(*[inst["x_true"].data_ptr() for inst in instances]) if has_xt else None
        o = L.sgks_options()
        o.max_iters, o.ell, o.n_refine, o.zeta, o.cgs_passes = max_iters, ell, n_refine, zeta, cgs_passes
        o.precision = PRECISIONS[precision]
        o.sketch_kind = L.SGKS_SKETCH_SPARSE_SIGN
        o.flags = (L.SGKS_FLAG_AUTOTUNE if autotune else 0) | (0 if tiles else L.SGKS_FLAG_NO_TILES)
        self.max_iters = max_iters
        dev = instances[0]["b"].device
        self.device = dev
        self._stream = torch.cuda.current_stream(dev).cuda_stream if stream is None else stream
        h = C.c_void_p()
        rc = self._lib.sgks_batch_create(C.byref(h), k, self._adesc, self._rdesc, self._b, self._lam, self._xt,
                                         int(sketch_rows), int(seed), C.byref(o), C.c_void_p(self._stream))
        L.check_batch(rc, None)
        self._h = h

    def reset(self, bs):
        if len(bs) != self.count:
            raise ValueError("one b per instance")
        for i, b in enumerate(bs):
            _need_cuda(b, "b")
            self._keep[i][1] = b
        arr = (C.c_void_p * self.count)(*[b.data_ptr() for b in bs])
        L.check_batch(self._lib.sgks_batch_reset(self._h, arr), self._h)

    def step(self):
        L.check_batch(self._lib.sgks_batch_step(self._h), self._h)

    def solve(self, iters: int, tol: float = 0.0, x_out=None, history: bool = False):
        """Run iters iterations; x_out: None or a list of device tensors (None entries skipped).
        Returns one report dict per instance."""
        k = self.count
        reps = (L.sgks_report * k)()
        hist = []
        if history:
            for i in range(k):
                rc_arr, rre_arr = (C.c_double * max(iters, 1))(), (C.c_double * max(iters, 1))()
                reps[i].rc = C.cast(rc_arr, C.POINTER(C.c_double))
                reps[i].rre = C.cast(rre_arr, C.POINTER(C.c_double))
                hist.append((rc_arr, rre_arr))
        xo = None
        if x_out is not None:
            for t in x_out:
                _need_cuda(t, "x_out")
            xo = (C.c_void_p * k)(*[None if t is None else t.data_ptr() for t in x_out])
        L.check_batch(self._lib.sgks_batch_solve(self._h, int(iters), float(tol), xo, reps), self._h)
        out = []
        for i in range(k):
            r = reps[i]
            d = dict(iters_done=r.iters_done, status=r.status, d=r.subspace_dim, rc_last=r.rc_last,
                     rre_last=r.rre_last, rre0=r.rre0)
            if history:
                d["rc"] = list(hist[i][0][:r.iters_done])
                d["rre"] = list(hist[i][1][:r.iters_done])
            out.append(d)
        return out

    def x(self, which=None):
        """Current iterates x_k (list of device tensors): of every instance, or of the instances
        listed in `which` (None in the other places of the list)."""
        pick = set(range(self.count)) if which is None else set(which)
        xs = [torch.empty(n, dtype=self.dtype, device=self.device) if i in pick else None
              for i, n in enumerate(self.n)]
        arr = (C.c_void_p * self.count)(*[t.data_ptr() if t is not None else None for t in xs])
        L.check_batch(self._lib.sgks_batch_get_x(self._h, arr), self._h)
        return xs

    def status(self):
        codes = (C.c_int32 * self.count)()
        L.check_batch(self._lib.sgks_batch_status(self._h, codes), self._h)
        return list(codes)

    def profile(self, iters: int):
        """Per-kernel CUDA-event timing of `iters` eager iterations (sgks_batch_profile_steps)."""
        n = L.SGKS_BATCH_PROFILE_CLASSES
        ms, cnt = (C.c_double * n)(), (C.c_int64 * n)()
        L.check_batch(self._lib.sgks_batch_profile_steps(self._h, int(iters), ms, cnt), self._h)
        return {L.BATCH_PROFILE_CLASS_NAMES[i]: dict(ms=ms[i], launches=cnt[i]) for i in range(n)}

    def config(self, group: int = 0) -> str:
        """The tile configuration the autotuner chose for a group ("" when not tuned)."""
        c = self._lib.sgks_batch_config(self._h, int(group))
        return c.decode() if c else ""

    def layout(self):
        g, sz = (C.c_int32 * self.count)(), (C.c_int32 * self.count)()
        ng = L.check_batch(self._lib.sgks_batch_layout(self._h, g, sz), self._h)
        return ng, list(g), list(sz)

    def close(self):
        if getattr(self, "_h", None):
            self._lib.sgks_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class SGKSFunction(torch.autograd.Function):
    """x_K(b, lambda) of a recording Solver as a differentiable torch function.

    forward(b, lam, solver, iters): sets lambda if it changed, resets the solver with b, runs
    iters iterations and returns a copy of x_K.  backward: the reverse sweep of the library
    (sgks_backward) gives dl/db and dl/dlambda.  The solver keeps the state of its last forward,
    so each forward must be followed by its backward before the solver is used again.
    """

    @staticmethod
    def forward(ctx, b, lam, solver, iters):
        lv = float(lam)
        if lv != solver.lam:
            solver.set_lambda(lv)
        solver.reset(b.detach().contiguous())
        solver.solve(int(iters))
        ctx.solver = solver
        ctx.lam_meta = (lam.dtype, lam.device) if torch.is_tensor(lam) else None
        return solver.x().clone()

    @staticmethod
    def backward(ctx, gx):
        gb, gl = ctx.solver.backward(gx.detach().to(ctx.solver.dtype).contiguous())
        glam = None
        if ctx.lam_meta is not None:
            glam = torch.tensor(gl, dtype=ctx.lam_meta[0], device=ctx.lam_meta[1])
        return gb, glam, None, None


def solve_differentiable(solver, b, lam, iters):
    """x_K = SGKSFunction.apply(b, lam, solver, iters) (lam a 0-dim tensor to get dl/dlambda)."""
    return SGKSFunction.apply(b, lam, solver, iters)


def kernel_launches() -> int:
    """Kernel launches enqueued by the library in this process (sgks_kernel_launches)."""
    return int(L.load().sgks_kernel_launches())


def sparse_sign_rows(seed: int, stream_id: int, h: int, s: int, zeta: int, device="cuda"):
    """Device-generated sparse-sign positions (rows[h, zeta] int32) and negative flags (uint8)."""
    lib = L.load()
    rows = torch.empty((h, zeta), dtype=torch.int32, device=device)
    neg = torch.empty((h, zeta), dtype=torch.uint8, device=device)
    st = torch.cuda.current_stream(rows.device).cuda_stream
    L.check(lib.sgks_sparse_sign_rows(int(seed), int(stream_id), int(h), int(s), int(zeta), _ptr(rows), _ptr(neg),
                                      C.c_void_p(st)))
    return rows, neg


def device_inputs(problem, precision: Optional[str] = None, device="cuda", transpose: bool = True):
    """Copy a problem description (fields as in workloads.Problem: A, L, b, x_true, lam, sketch,
    iters, n_refine) to the device and return the keyword arguments of ``Solver``.

    A's values, the PSF and the dense matrix are passed as float32 (the problem data are
    float32-representable); b and x_true in the solver precision; a Gaussian sketch in float64.
    """
    import numpy as np

    prec = precision or problem.precision
    dt = io_dtype(prec)
    A = problem.A
    if A.kind == "csr":
        op = CSR(torch.from_numpy(np.ascontiguousarray(A.row_ptr)).to(device),
                 torch.from_numpy(np.ascontiguousarray(A.col)).to(device),
                 torch.from_numpy(np.ascontiguousarray(A.val, dtype=np.float32)).to(device), A.m, A.n)
        if transpose:
            op.transposed()
    elif A.kind == "dense":
        op = Dense(torch.from_numpy(np.ascontiguousarray(A.dense, dtype=np.float32)).to(device))
    elif A.kind == "conv2d":
        op = Conv2D(torch.from_numpy(np.ascontiguousarray(A.psf, dtype=np.float32)).to(device), A.nx, A.ny)
    else:
        raise ValueError(A.kind)
    Lr = problem.L
    reg = Reg(Lr.kind, Lr.nx, Lr.ny, Lr.nt)
    sk = problem.sketch
    kw = dict(A=op, reg=reg, b=torch.from_numpy(np.asarray(problem.b)).to(device, dt), lam=float(problem.lam),
              sketch_rows=int(sk.s), seed=int(sk.seed), max_iters=int(problem.iters),
              n_refine=int(problem.n_refine), precision=prec, sketch=sk.kind, zeta=int(sk.zeta),
              x_true=torch.from_numpy(np.asarray(problem.x_true)).to(device, dt))
    if sk.kind == "gaussian":
        kw["gauss_SA"] = torch.from_numpy(np.ascontiguousarray(sk.SA, dtype=np.float64)).to(device)
        kw["gauss_SL"] = torch.from_numpy(np.ascontiguousarray(sk.SL, dtype=np.float64)).to(device)
    if sk.kind == "srtt":
        kw["srtt"] = tuple(torch.from_numpy(np.ascontiguousarray(a)).to(device)
                           for a in (sk.signs_A.astype(np.int8), sk.rows_A.astype(np.int32),
                                     sk.signs_L.astype(np.int8), sk.rows_L.astype(np.int32)))
    return kw
