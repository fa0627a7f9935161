"""Python binding of libcondipm (condensed-space IPM KKT solves on GB300).

Argument marshalling only: every step runs in the library's CUDA kernels.  Tensors are
passed by device pointer on torch's current CUDA stream.  The extension must be built
(``__graft_entry__.build()``); there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import LIB

_lib = None

IPM_OK, IPM_ERR_NOT_PD, IPM_ERR_CG_MAXIT, IPM_ERR_NONFINITE = 0, 1, 2, 3
IPM_ERR_BAD_ARG, IPM_ERR_OOM, IPM_ERR_CUDA = -1, -2, -3
IPM_ERR_TIMEOUT, IPM_ERR_RESTORATION, IPM_ERR_INERTIA, IPM_ERR_MAXITER = 4, 5, 6, 7
IPM_ERR_INFEASIBLE = 8

P = ctypes.c_void_p
I = ctypes.c_int
D = ctypes.c_double
I64 = ctypes.c_int64

_SIGS = {
    "ipm_last_error_message": (ctypes.c_char_p, []),
    "ipm_symbolic": (I, [I, I, P, P, I, P, P, I, P, P]),
    "ipm_symbolic_relaxed": (I, [I, I, P, P, I, P, P, I, I, I, P, P]),
    "ipm_symbolic_info": (I, [P, P, P, P, P, P, P]),
    "ipm_launch_count": (ctypes.c_longlong, []),
    "ipm_symbolic_export": (I, [P, P, P, P, P, P]),
    "ipm_symbolic_export_panels": (I, [P, P, P, P]),
    "ipm_symbolic_destroy": (None, [P]),
    "ipm_num_create": (I, [P, I, P]),
    "ipm_num_destroy": (None, [P]),
    "ipm_num_export": (I, [P, P]),
    "ipm_num_status": (I, [P, P]),
    "ipm_num_info": (I, [P, P, P]),
    "ipm_set_spin_limit": (I, [ctypes.c_longlong]),
    "ipm_debug_add_dependency": (I, [P, I, I]),
    "ipm_debug_poison_allocations": (I, [I]),
    "ipm_condense": (I, [P, P, P, P, P, P, D, P]),
    "ipm_factor": (I, [P, P, P, P]),
    "ipm_solve": (I, [P, P, P, P, I, P]),
    "ipm_solve_noalloc": (I, [P, P, P, P, P, P]),
    "ipm_aug_solve": (I, [P, P, P, P, P, P, D, P, P, P, P, I, D, P, P, P]),
    "hykkt_cg": (I, [P, P, I, P, P, D, P, P, D, I, P, P, P, P, P, P]),
    "ipm_opf_create": (I, [I, I, I] + [P] * 13 + [P, P]),
    "ipm_opf_create_flow": (I, [I, I, I] + [P] * 13 + [P, P]),
    "ipm_opf_info": (I, [P, P, P, P, P, P]),
    "ipm_opf_patterns": (I, [P, P, P, P, P]),
    "ipm_opf_eval": (I, [P, P, P, P, D, P, P, P, P, P, P, P]),
    "ipm_opf_destroy": (None, [P]),
    "ipm_state_create": (I, [P, P, P, P]),
    "ipm_state_create_at": (I, [P, P, P, P, P]),
    "ipm_step": (I, [P, P]),
    "ipm_state_export": (I, [P, P, P]),
    "ipm_state_save": (I, [P, P, I64, P]),
    "ipm_state_load": (I, [P, P, I64]),
    "ipm_state_export_kkt": (I, [P] * 11),
    "ipm_state_destroy": (None, [P]),
    "ipm_batch_create": (I, [I, P, P, P, P]),
    "ipm_batch_info": (I, [P, P, P, P]),
    "ipm_batch_reset": (I, [P]),
    "ipm_batch_run": (I, [P, I, I, I]),
    "ipm_batch_results": (I, [P, P, P, P, P, P, P]),
    "ipm_batch_cg_iters": (I, [P, P]),
    "ipm_batch_resto_counts": (I, [P, P, P]),
    "ipm_batch_solve_info": (I, [P, P, P, P, P, P, P]),
    "ipm_batch_set_tail": (I, [P, I, I]),
    "ipm_batch_autotune": (I, [P, I, I, P, P, P, P]),
    "ipm_batch_export": (I, [P, I, P]),
    "ipm_batch_sweeps": (I, [P]),
    "ipm_batch_pause_at": (I, [P, I]),
    "ipm_batch_set_shape": (I, [P, I, I, I, I, P]),
    "ipm_batch_resume": (I, [P]),
    "ipm_batch_export_kkt": (I, [P, I] + [P] * 10),
    "ipm_batch_destroy": (None, [P]),
    "ipm_batch_export_all": (I, [P, P]),
    "ipm_batch_set_timing": (I, [P, I]),
    "ipm_batch_kernel_time": (I, [P, P, P, P]),
    "ipm_batch_work": (I, [P, P, P, P]),
    "ipm_opf_set_loads": (I, [P, P, P, P]),
    "ipm_batch_state_rows": (I, [P, P, I64, P]),
    "ipm_batch_warm_start": (I, [P, P, I64, P, P, P]),
    "mlp_create": (I, [I, P, I, P]),
    "mlp_param_count": (I, [P, P]),
    "mlp_set_params": (I, [P, P]),
    "mlp_get_params": (I, [P, P]),
    "mlp_get_grads": (I, [P, P]),
    "mlp_forward": (I, [P, P, I, P, P]),
    "mlp_loss_backward": (I, [P, P, I, P, P]),
    "mlp_adam_step": (I, [P, ctypes.c_float, ctypes.c_float, ctypes.c_float, ctypes.c_float, I, P]),
    "mlp_gather_rows": (I, [I, I, P, P, P, P]),
    "mlp_col_stats": (I, [I, I, P, P, P, ctypes.c_float, P]),
    "mlp_normalize": (I, [I, I, P, P, P, P, P]),
    "mlp_destroy": (None, [P]),
}


class IpmOptions(ctypes.Structure):
    _fields_ = [("kkt", ctypes.c_int), ("tol", ctypes.c_double), ("gamma", ctypes.c_double),
                ("tau", ctypes.c_double), ("mu0", ctypes.c_double), ("cg_rtol", ctypes.c_double),
                ("max_refine", ctypes.c_int), ("cg_maxit", ctypes.c_int),
                ("precision", ctypes.c_int), ("sn_relax_w", ctypes.c_int),
                ("sn_relax_den", ctypes.c_int), ("no_resto", ctypes.c_int)]


class IpmIterInfo(ctypes.Structure):
    _fields_ = [("k", ctypes.c_int), ("status", ctypes.c_int), ("mu", ctypes.c_double),
                ("kkt_err", ctypes.c_double), ("alpha", ctypes.c_double),
                ("delta_w", ctypes.c_double), ("obj", ctypes.c_double), ("eta", ctypes.c_double),
                ("theta", ctypes.c_double), ("n_factor", ctypes.c_int), ("cg_iters", ctypes.c_int),
                ("refine_steps", ctypes.c_int), ("ls_steps", ctypes.c_int),
                ("precision", ctypes.c_int), ("gamma", ctypes.c_double),
                ("pcg_iters", ctypes.c_int), ("resto", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class CondipmError(RuntimeError):
    pass


def lib():
    """Loads libcondipm.so; raises if it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB):
            raise CondipmError(f"{LIB} is missing: build it with __graft_entry__.build()")
        L = ctypes.CDLL(LIB)
        for name, (res, args) in _SIGS.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def launch_count() -> int:
    """Kernels launched so far by the library's numeric entry points."""
    return int(lib().ipm_launch_count())


def exported_symbols():
    return list(_SIGS)


def _check(rc, name):
    if rc < 0:
        msg = lib().ipm_last_error_message()
        raise CondipmError(f"{name} failed ({rc}): {msg.decode() if msg else ''}")
    return rc


def _ptr(t, dtype=None):
    import torch
    if t is None:
        return None
    assert t.is_cuda and t.is_contiguous(), "expected a contiguous CUDA tensor"
    if dtype is not None:
        assert t.dtype == dtype, f"expected {dtype}, got {t.dtype}"
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    import torch
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Symbolic:
    """ipm_symbolic handle for one (J, W-lower) sparsity pattern (int32 CUDA tensors)."""

    def __init__(self, n, m, J_rowptr, J_colind, W_rowptr, W_colind, stream=None, relax=(8, 5)):
        import torch
        h = ctypes.c_void_p()
        _check(lib().ipm_symbolic_relaxed(n, m, _ptr(J_rowptr, torch.int32),
                                          _ptr(J_colind, torch.int32), int(J_colind.numel()),
                                          _ptr(W_rowptr, torch.int32), _ptr(W_colind, torch.int32),
                                          int(W_colind.numel()), int(relax[0]), int(relax[1]),
                                          _stream(stream), ctypes.byref(h)), "ipm_symbolic")
        self.h = h
        self.n, self.m = n, m
        nk, ns, nnz, plen, nl, fl = I64(), I(), I64(), I64(), I(), D()
        _check(lib().ipm_symbolic_info(h, ctypes.byref(nk), ctypes.byref(ns), ctypes.byref(nnz),
                                       ctypes.byref(plen), ctypes.byref(nl), ctypes.byref(fl)),
               "ipm_symbolic_info")
        self.nnz_k = nk.value
        self.nsuper, self.nnz_offdiag, self.panel_len = ns.value, nnz.value, plen.value
        self.nlevels, self.flops = nl.value, fl.value

    def export(self):
        n = self.n
        perm = np.zeros(n, np.int32)
        parent = np.zeros(n, np.int32)
        sptr = np.zeros(self.nsuper + 1, np.int32)
        colptr = np.zeros(n + 1, np.int64)
        rowind = np.zeros(max(self.nnz_offdiag, 1), np.int32)
        c = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        _check(lib().ipm_symbolic_export(self.h, c(perm), c(parent), c(sptr), c(colptr), c(rowind)),
               "ipm_symbolic_export")
        return dict(perm=perm, parent=parent, sptr=sptr, colptr=colptr,
                    rowind=rowind[:self.nnz_offdiag])

    def export_panels(self):
        srow_ptr = np.zeros(self.nsuper + 1, np.int32)
        lptr = np.zeros(self.nsuper + 1, np.int64)
        c = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        _check(lib().ipm_symbolic_export_panels(self.h, c(srow_ptr), None, c(lptr)), "export_panels")
        srow = np.zeros(max(int(srow_ptr[-1]), 1), np.int32)
        _check(lib().ipm_symbolic_export_panels(self.h, None, c(srow), None), "export_panels")
        return srow_ptr, srow[:int(srow_ptr[-1])], lptr

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.ipm_symbolic_destroy(self.h)
            self.h = None


class Numeric:
    """ipm_num handle: panel storage + workspaces for one Symbolic."""

    def __init__(self, sym: Symbolic, precision: int = 64):
        h = ctypes.c_void_p()
        _check(lib().ipm_num_create(sym.h, precision, ctypes.byref(h)), "ipm_num_create")
        self.h, self.sym = h, sym

    def export(self):
        out = np.zeros(max(self.sym.panel_len, 1), np.float64)
        _check(lib().ipm_num_export(self.h, out.ctypes.data_as(ctypes.c_void_p)), "ipm_num_export")
        return out[:self.sym.panel_len]

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.ipm_num_destroy(self.h)
            self.h = None


def ipm_num_info(num):
    prec, its = I(), I()
    _check(lib().ipm_num_info(num.h, ctypes.byref(prec), ctypes.byref(its)), "ipm_num_info")
    return prec.value, its.value


def ipm_num_status(num):
    st = I()
    _check(lib().ipm_num_status(num.h, ctypes.byref(st)), "ipm_num_status")
    return st.value


def ipm_set_spin_limit(polls):
    return _check(lib().ipm_set_spin_limit(int(polls)), "ipm_set_spin_limit")


def ipm_debug_poison_allocations(on=True):
    """While on, floating-point buffers the library allocates start as NaN (debugging aid)."""
    return _check(lib().ipm_debug_poison_allocations(int(bool(on))), "ipm_debug_poison_allocations")


def ipm_debug_add_dependency(sym, supernode, extra=1):
    return _check(lib().ipm_debug_add_dependency(sym.h, int(supernode), int(extra)),
                  "ipm_debug_add_dependency")


def ipm_condense(sym, num, W_val, sigma_x, J_val, d_row, delta_w, stream=None):
    rc = _check(lib().ipm_condense(sym.h, num.h, _ptr(W_val), _ptr(sigma_x), _ptr(J_val),
                                   _ptr(d_row), float(delta_w), _stream(stream)), "ipm_condense")
    # the library keeps these pointers for the FP64 products of later solves on this handle
    # (refinement, the FP32 factor's CG): the tensors live as long as the handle refers to them
    num._condense_inputs = (W_val, sigma_x, J_val, d_row)
    return rc


def ipm_factor(sym, num, d_info, stream=None):
    return _check(lib().ipm_factor(sym.h, num.h, _ptr(d_info), _stream(stream)), "ipm_factor")


def ipm_solve(sym, num, b, x, stream=None):
    """x = K^{-1} b; b, x: [n] or [nrhs, n] contiguous float64 CUDA tensors (each row one
    right-hand side: the C-ABI's column-major n x nrhs)."""
    nrhs = 1 if b.dim() == 1 else int(b.shape[0])
    if tuple(x.shape) != tuple(b.shape) or b.shape[-1] != sym.n:
        raise ValueError("ipm_solve: b and x must both be [n] or [nrhs, n]")
    return _check(lib().ipm_solve(sym.h, num.h, _ptr(b), _ptr(x), nrhs, _stream(stream)),
                  "ipm_solve")


def ipm_solve_noalloc(sym, num, b, x, d_status=None, stream=None):
    """Solve with the library's static scratch instead of the handle's workspace (no allocation)."""
    return _check(lib().ipm_solve_noalloc(sym.h, num.h, _ptr(b), _ptr(x), _ptr(d_status),
                                          _stream(stream)), "ipm_solve_noalloc")


def ipm_aug_solve(sym, num, W_val, sigma_x, J_val, d_row, delta_w, a, b, dx, dz, d_eta, d_steps,
                  max_refine=10, tol=1e-10, stream=None):
    return _check(lib().ipm_aug_solve(sym.h, num.h, _ptr(W_val), _ptr(sigma_x), _ptr(J_val),
                                      _ptr(d_row), float(delta_w), _ptr(a), _ptr(b), _ptr(dx),
                                      _ptr(dz), int(max_refine), float(tol), _ptr(d_eta),
                                      _ptr(d_steps), _stream(stream)), "ipm_aug_solve")


def hykkt_cg(sym, num, m_e, J_val, d_row, gamma, a, b, dx, dy, dz, rtol=1e-10, maxit=None,
             stream=None):
    its, rel = I(), D()
    maxit = max(m_e, 1) if maxit is None else maxit
    rc = _check(lib().hykkt_cg(sym.h, num.h, int(m_e), _ptr(J_val), _ptr(d_row), float(gamma),
                               _ptr(a), _ptr(b), float(rtol), int(maxit), _ptr(dx), _ptr(dy),
                               _ptr(dz), ctypes.byref(its), ctypes.byref(rel), _stream(stream)),
                "hykkt_cg")
    return rc, its.value, rel.value


class Opf:
    """ipm_opf handle for one synthetic grid (``synth.Grid``); patterns as int32 CUDA tensors."""

    def __init__(self, grid, stream=None, form="compact"):
        """form "compact" (x = [V | theta | Pg | Qg]) or "flow" (plus branch-flow variables)."""
        import torch
        c = lambda a, dt: np.ascontiguousarray(a, dtype=dt)
        self._keep = [c(grid.f_bus, np.int32), c(grid.t_bus, np.int32), c(grid.r, np.float64),
                      c(grid.x, np.float64), c(grid.b, np.float64), c(grid.rate, np.float64),
                      c(grid.pd, np.float64), c(grid.qd, np.float64), c(grid.gen_bus, np.int32),
                      c(grid.c2, np.float64), c(grid.c1, np.float64)]
        lo, hi = grid.bounds()
        self._keep += [c(lo, np.float64), c(hi, np.float64)]
        ptrs = [a.ctypes.data_as(ctypes.c_void_p) for a in self._keep]
        h = ctypes.c_void_p()
        create = lib().ipm_opf_create_flow if form == "flow" else lib().ipm_opf_create
        _check(create(grid.nb, grid.nbr, grid.ng, *ptrs, _stream(stream), ctypes.byref(h)),
               "ipm_opf_create")
        self.h = h
        n, me, mi, nj, nw = I(), I(), I(), I(), I()
        _check(lib().ipm_opf_info(h, *(ctypes.byref(v) for v in (n, me, mi, nj, nw))), "ipm_opf_info")
        self.n, self.m_e, self.m_i, self.nnzJ, self.nnzW = n.value, me.value, mi.value, nj.value, nw.value
        dev = dict(dtype=torch.int32, device="cuda")
        self.J_rowptr = torch.empty(self.m_e + self.m_i + 1, **dev)
        self.J_colind = torch.empty(max(self.nnzJ, 1), **dev)
        self.W_rowptr = torch.empty(self.n + 1, **dev)
        self.W_colind = torch.empty(max(self.nnzW, 1), **dev)
        _check(lib().ipm_opf_patterns(h, _ptr(self.J_rowptr), _ptr(self.J_colind), _ptr(self.W_rowptr),
                                      _ptr(self.W_colind)), "ipm_opf_patterns")
        self.J_colind = self.J_colind[:self.nnzJ]
        self.W_colind = self.W_colind[:self.nnzW]

    def set_loads(self, pd, qd, stream=None):
        """New loads (numpy float64 host arrays or CUDA tensors, nb values each)."""
        ptr = lambda a: a.ctypes.data_as(ctypes.c_void_p) if isinstance(a, np.ndarray) else _ptr(a)
        _check(lib().ipm_opf_set_loads(self.h, ptr(pd), ptr(qd), _stream(stream)),
               "ipm_opf_set_loads")

    def eval(self, x, y, z, sigma_f, f, grad, g, h, J_val, W_val, stream=None):
        return _check(lib().ipm_opf_eval(self.h, _ptr(x), _ptr(y), _ptr(z), float(sigma_f), _ptr(f),
                                         _ptr(grad), _ptr(g), _ptr(h), _ptr(J_val), _ptr(W_val),
                                         _stream(stream)), "ipm_opf_eval")

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.ipm_opf_destroy(self.h)
            self.h = None


class IpmState:
    """GPU interior-point iterate for an ``Opf`` problem (ipm_state_create / ipm_step)."""

    def __init__(self, opf, kkt="lifted", tol=1e-6, gamma=1e6, tau=0.0, mu0=0.1, cg_rtol=1e-10,
                 max_refine=10, cg_maxit=0, precision=64, stream=None, relax=(0, 0), x0=None,
                 restoration=True):
        """x0: optional starting point (n host values, pushed inside the bounds;
        ipm_state_create_at), else the flat start.  restoration=False: a failed line search
        ends the solve (IPM_ERR_RESTORATION) instead of entering the restoration phase."""
        self.opf = opf
        o = IpmOptions({"lifted": 0, "hykkt": 1, "regularized": 2}[kkt], tol, gamma, tau, mu0,
                       cg_rtol, max_refine, cg_maxit, precision, int(relax[0]), int(relax[1]),
                       int(not restoration))
        h = ctypes.c_void_p()
        if x0 is None:
            _check(lib().ipm_state_create(opf.h, ctypes.byref(o), _stream(stream),
                                          ctypes.byref(h)), "ipm_state_create")
        else:
            x0 = np.ascontiguousarray(x0, dtype=np.float64)
            if x0.shape != (opf.n,):
                raise ValueError(f"x0 must hold n = {opf.n} values")
            _check(lib().ipm_state_create_at(opf.h, ctypes.byref(o),
                                             x0.ctypes.data_as(ctypes.c_void_p), _stream(stream),
                                             ctypes.byref(h)), "ipm_state_create_at")
        self.h = h

    def step(self):
        info = IpmIterInfo()
        _check(lib().ipm_step(self.h, ctypes.byref(info)), "ipm_step")
        return info

    def x(self):
        out = np.zeros(self.opf.n)
        _check(lib().ipm_state_export(self.h, out.ctypes.data_as(ctypes.c_void_p), None), "export")
        return out

    def save(self):
        """Checkpoint of the iteration (ipm_state_save) as a float64 array."""
        n = I64()
        _check(lib().ipm_state_save(self.h, None, 0, ctypes.byref(n)), "ipm_state_save")
        buf = np.zeros(n.value)
        _check(lib().ipm_state_save(self.h, buf.ctypes.data_as(ctypes.c_void_p), n.value,
                                    ctypes.byref(n)), "ipm_state_save")
        return buf

    def load(self, buf):
        """Continue from a checkpoint of save() (ipm_state_load)."""
        buf = np.ascontiguousarray(buf, dtype=np.float64)
        _check(lib().ipm_state_load(self.h, buf.ctypes.data_as(ctypes.c_void_p), buf.size),
               "ipm_state_load")

    def objective(self):
        v = D()
        _check(lib().ipm_state_export(self.h, None, ctypes.byref(v)), "export")
        return v.value

    def export_kkt(self):
        """The augmented KKT system of the last step and its refined solution
        (ipm_state_export_kkt), as host arrays."""
        o = self.opf
        m = o.m_e + o.m_i
        out = dict(W_val=np.zeros(o.nnzW), sigma=np.zeros(o.n), J_val=np.zeros(o.nnzJ),
                   d_row=np.zeros(m), a=np.zeros(o.n), b=np.zeros(m), dx=np.zeros(o.n),
                   dyz=np.zeros(m))
        dw, me = D(), I()
        p = lambda k: out[k].ctypes.data_as(ctypes.c_void_p)
        _check(lib().ipm_state_export_kkt(self.h, p("W_val"), p("sigma"), p("J_val"), p("d_row"),
                                          ctypes.byref(dw), p("a"), p("b"), p("dx"), p("dyz"),
                                          ctypes.byref(me)), "ipm_state_export_kkt")
        out["delta_w"], out["m_e"] = dw.value, me.value
        return out

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.ipm_state_destroy(self.h)
            self.h = None


def ipm_solve_opf(opf, max_iter=3000, **opts):
    """Runs ipm_step until convergence, failure or max_iter iterations of the main problem
    (iterations of the restoration phase, bounded by the library, do not count); returns
    (status, iters, obj, history)."""
    st = IpmState(opf, **opts)
    hist = []
    status = 0
    main = 0
    while main <= max_iter:
        info = st.step()
        hist.append(info.as_dict())
        status = info.status
        if status != 0:
            break
        main += info.resto != 1
    iters = hist[-1]["k"]
    return dict(status=status, iters=iters, obj=st.objective(), x=st.x(), history=hist, state=st)


class Batch:
    """Batched interior-point solves over ``Opf`` handles (ipm_batch_*): one symbolic analysis
    per distinct pattern, every instance advanced by the same launches.  kkt: "lifted",
    "hykkt" (CG on the Schur complement of K_gamma) or "regularized".  precision 32 (lifted or
    regularized): FP32 factor and triangular solves inside FP64 refinement, each instance going
    to FP64 when its FP32 solve cannot reach a backward error of 1e-10."""

    def __init__(self, opfs, tol=1e-6, tau=0.0, mu0=0.1, max_refine=10, kkt="lifted", gamma=1e6,
                 cg_rtol=1e-10, cg_maxit=0, stream=None, relax=(0, 0), restoration=True,
                 precision=64):
        self.opfs = list(opfs)
        arr = (ctypes.c_void_p * len(self.opfs))(*[o.h.value for o in self.opfs])
        o = IpmOptions({"lifted": 0, "hykkt": 1, "regularized": 2}[kkt], tol, gamma, tau, mu0,
                       cg_rtol, max_refine, cg_maxit, int(precision), int(relax[0]),
                       int(relax[1]), int(not restoration))
        h = ctypes.c_void_p()
        _check(lib().ipm_batch_create(len(self.opfs), arr, ctypes.byref(o), _stream(stream),
                                      ctypes.byref(h)), "ipm_batch_create")
        self.h = h
        self.count = len(self.opfs)

    def info(self):
        npat, nbytes, nl = I(), I64(), I()
        _check(lib().ipm_batch_info(self.h, ctypes.byref(npat), ctypes.byref(nbytes),
                                    ctypes.byref(nl)), "ipm_batch_info")
        return dict(patterns=npat.value, device_bytes=nbytes.value, launches_per_sweep=nl.value)

    def reset(self):
        _check(lib().ipm_batch_reset(self.h), "ipm_batch_reset")

    def run(self, max_iter=3000, max_sweeps=None, use_graph=True):
        ms = 4 * max_iter + 100 if max_sweeps is None else max_sweeps
        _check(lib().ipm_batch_run(self.h, int(max_iter), int(ms), int(bool(use_graph))),
               "ipm_batch_run")

    def results(self):
        n = self.count
        st, it, nf, ls = (np.zeros(n, np.int32) for _ in range(4))
        obj, err = np.zeros(n), np.zeros(n)
        p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        _check(lib().ipm_batch_results(self.h, p(st), p(it), p(obj), p(err), p(nf), p(ls)),
               "ipm_batch_results")
        cg = np.zeros(n, np.int32)
        _check(lib().ipm_batch_cg_iters(self.h, p(cg)), "ipm_batch_cg_iters")
        rph, rit = np.zeros(n, np.int32), np.zeros(n, np.int32)
        _check(lib().ipm_batch_resto_counts(self.h, p(rph), p(rit)), "ipm_batch_resto_counts")
        return dict(status=st, iters=it, obj=obj, kkt_err=err, n_factor=nf, ls_steps=ls,
                    cg_iters=cg, resto_phases=rph, resto_iters=rit,
                    sweeps=lib().ipm_batch_sweeps(self.h))

    def solve_info(self):
        """Per instance (ipm_batch_solve_info): the factor precision used now (32 or 64), the
        iterations whose KKT solve used the FP32 factor, the iteration at which it went to FP64
        (-1: never), KKT solves finished, those above a backward error of 1e-10 and the
        largest final backward error."""
        n = self.count
        cur, it32, k64, ns, na = (np.zeros(n, np.int32) for _ in range(5))
        em = np.zeros(n)
        p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        _check(lib().ipm_batch_solve_info(self.h, p(cur), p(it32), p(k64), p(ns), p(na), p(em)),
               "ipm_batch_solve_info")
        return dict(current=cur, iters32=it32, k64=k64, solves=ns, above=na, eta_max=em)

    def autotune(self, sweeps=8):
        """Times the candidate launch shapes (ipm_batch_autotune) and keeps the fastest; every
        instance is back at its starting point afterwards.  Returns the candidates as dicts
        (cluster, threshold, blocks_per_instance, ms_per_sweep) and the chosen index."""
        cap = 64
        cfg = np.zeros(4 * cap, np.int32)
        ms = np.zeros(cap)
        n, best = I(), I()
        p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        _check(lib().ipm_batch_autotune(self.h, int(sweeps), cap, ctypes.byref(n), p(cfg), p(ms),
                                        ctypes.byref(best)), "ipm_batch_autotune")
        out = [dict(cluster=int(cfg[4 * k]), threshold=(float(cfg[4 * k + 1]) / cfg[4 * k + 2]
                                                         if cfg[4 * k + 2] else None),
                    blocks_per_instance=int(cfg[4 * k + 3]), ms_per_sweep=float(ms[k]))
               for k in range(min(n.value, cap))]
        return dict(candidates=out, best=best.value)

    def x_all(self, out=None):
        """Every instance's x, concatenated (one gather and one copy); out: float64 numpy array."""
        if out is None:
            out = np.zeros(sum(o.n for o in self.opfs))
        _check(lib().ipm_batch_export_all(self.h, out.ctypes.data_as(ctypes.c_void_p)),
               "ipm_batch_export_all")
        return out

    def set_timing(self, on=True):
        _check(lib().ipm_batch_set_timing(self.h, int(bool(on))), "ipm_batch_set_timing")

    def kernel_time(self):
        f, s_, n = D(), D(), I()
        _check(lib().ipm_batch_kernel_time(self.h, ctypes.byref(f), ctypes.byref(s_),
                                           ctypes.byref(n)), "ipm_batch_kernel_time")
        return dict(fact_ms=f.value, solve_ms=s_.value, sweeps=n.value)

    def work(self):
        n = self.count
        ff, cf, by = np.zeros(n), np.zeros(n), np.zeros(n)
        p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
        _check(lib().ipm_batch_work(self.h, p(ff), p(cf), p(by)), "ipm_batch_work")
        return dict(factor_flops=ff, condense_flops=cf, bytes=by)

    def state_rows(self, out=None):
        """Every instance's (x, log s, log v, log zl, log zu[, y]) as a float32 CUDA matrix (y:
        HyKKT and dual-regularized batches)."""
        import torch
        w = I()
        _check(lib().ipm_batch_state_rows(self.h, None, 0, ctypes.byref(w)), "ipm_batch_state_rows")
        if out is None:
            out = torch.empty(self.count, w.value, dtype=torch.float32, device="cuda")
        _check(lib().ipm_batch_state_rows(self.h, _ptr(out), out.stride(0), None),
               "ipm_batch_state_rows")
        return out

    def warm_start(self, pred, mean=None, std=None):
        """Start every instance from the predicted rows (after reset); returns the used flags."""
        used = np.zeros(self.count, np.int32)
        _check(lib().ipm_batch_warm_start(self.h, _ptr(pred), pred.stride(0), _ptr(mean),
                                          _ptr(std), used.ctypes.data_as(ctypes.c_void_p)),
               "ipm_batch_warm_start")
        return used

    def x(self, i):
        out = np.zeros(self.opfs[i].n)
        _check(lib().ipm_batch_export(self.h, int(i), out.ctypes.data_as(ctypes.c_void_p)),
               "ipm_batch_export")
        return out

    def set_tail(self, active_max, cluster=8):
        """In batches of more than active_max instances, once at most active_max remain, sweeps
        hold more inertia and line-search rounds and (cluster > 0) run every instance on
        clusters (ipm_batch_set_tail; active_max 0 disables)."""
        _check(lib().ipm_batch_set_tail(self.h, int(active_max), int(cluster)),
               "ipm_batch_set_tail")

    def set_shape(self, cluster, big_num, big_den, gx):
        """Launch shape (ipm_batch_set_shape); returns the number of instances on clusters."""
        nb = I()
        _check(lib().ipm_batch_set_shape(self.h, int(cluster), int(big_num), int(big_den), int(gx),
                                         ctypes.byref(nb)), "ipm_batch_set_shape")
        return nb.value

    def pause_at(self, k):
        """Hold every instance after the KKT solve of its iteration k (-1: none)."""
        _check(lib().ipm_batch_pause_at(self.h, int(k)), "ipm_batch_pause_at")

    def resume(self):
        _check(lib().ipm_batch_resume(self.h), "ipm_batch_resume")

    def export_kkt(self, i):
        """Instance i's KKT system and refined solution while it is held (dict of host arrays,
        the layout of IpmState.export_kkt)."""
        o = self.opfs[i]
        m = o.m_e + o.m_i
        out = dict(W_val=np.zeros(o.nnzW), sigma=np.zeros(o.n), J_val=np.zeros(o.nnzJ),
                   d_row=np.zeros(m), a=np.zeros(o.n), b=np.zeros(m), dx=np.zeros(o.n),
                   dyz=np.zeros(m))
        dw, me = D(), I()
        p = lambda k: out[k].ctypes.data_as(ctypes.c_void_p)
        _check(lib().ipm_batch_export_kkt(self.h, int(i), p("W_val"), p("sigma"), p("J_val"),
                                          p("d_row"), ctypes.byref(dw), p("a"), p("b"), p("dx"),
                                          p("dyz"), ctypes.byref(me)), "ipm_batch_export_kkt")
        out["delta_w"], out["m_e"] = dw.value, me.value
        return out

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.ipm_batch_destroy(self.h)
            self.h = None


class MLP:
    """BF16 multilayer perceptron on the project's own kernels (mlp_*): GELU hidden layers,
    linear output, MSE loss, Adam."""

    def __init__(self, dims, max_batch):
        self.dims = [int(d) for d in dims]
        arr = (ctypes.c_int * len(self.dims))(*self.dims)
        h = ctypes.c_void_p()
        _check(lib().mlp_create(len(self.dims) - 1, arr, int(max_batch), ctypes.byref(h)),
               "mlp_create")
        self.h = h
        self.max_batch = int(max_batch)
        c = I64()
        _check(lib().mlp_param_count(h, ctypes.byref(c)), "mlp_param_count")
        self.nparams = c.value
        import torch
        self._loss = torch.zeros(1, dtype=torch.float32, device="cuda")
        self.t = 0

    def set_params(self, flat):
        a = np.ascontiguousarray(flat, dtype=np.float32)
        assert a.size == self.nparams
        _check(lib().mlp_set_params(self.h, a.ctypes.data_as(ctypes.c_void_p)), "mlp_set_params")
        self.t = 0

    def get_params(self):
        a = np.zeros(self.nparams, np.float32)
        _check(lib().mlp_get_params(self.h, a.ctypes.data_as(ctypes.c_void_p)), "mlp_get_params")
        return a

    def get_grads(self):
        a = np.zeros(self.nparams, np.float32)
        _check(lib().mlp_get_grads(self.h, a.ctypes.data_as(ctypes.c_void_p)), "mlp_get_grads")
        return a

    def forward(self, X, Y=None):
        _check(lib().mlp_forward(self.h, _ptr(X), X.shape[0], _ptr(Y), None), "mlp_forward")
        return Y

    def loss_backward(self, T):
        _check(lib().mlp_loss_backward(self.h, _ptr(T), T.shape[0], _ptr(self._loss), None),
               "mlp_loss_backward")
        return self._loss

    def adam(self, lr, b1=0.9, b2=0.999, eps=1e-8):
        self.t += 1
        _check(lib().mlp_adam_step(self.h, float(lr), float(b1), float(b2), float(eps), self.t,
                                   None), "mlp_adam_step")

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.mlp_destroy(self.h)
            self.h = None


def gather_rows(idx, src, out):
    _check(lib().mlp_gather_rows(idx.shape[0], src.shape[1], _ptr(idx), _ptr(src), _ptr(out), None),
           "mlp_gather_rows")
    return out


def col_stats(src, floor_std=1e-3):
    import torch
    mean = torch.empty(src.shape[1], dtype=torch.float32, device="cuda")
    std = torch.empty_like(mean)
    _check(lib().mlp_col_stats(src.shape[0], src.shape[1], _ptr(src), _ptr(mean), _ptr(std),
                               float(floor_std), None), "mlp_col_stats")
    return mean, std


def normalize(src, mean, std, out=None):
    out = src if out is None else out
    _check(lib().mlp_normalize(src.shape[0], src.shape[1], _ptr(src), _ptr(mean), _ptr(std),
                               _ptr(out), None), "mlp_normalize")
    return out

