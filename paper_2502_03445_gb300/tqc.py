"""Thin ctypes binding of libtqc (argument marshalling only).

Every step of the reconstruction runs in the library's CUDA kernels; this
module only converts Python objects to the C ABI declared in
``include/tqc.h``.  There is no Python or CPU fallback: if the library is
missing, importing :func:`lib` raises.

Device memory and streams come from PyTorch (``torch.Tensor.data_ptr()``,
``torch.cuda.current_stream().cuda_stream``)."""
from __future__ import annotations

import ctypes
import json
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libtqc.so")

OK, ERR_INVALID, ERR_OOM, ERR_CUDA, ERR_TIMEOUT, ERR_UNSUPPORTED = range(6)
F64, F32 = 0, 1
PREC_FP32, PREC_TF32, PREC_BF16, PREC_BF16X3, PREC_AUTO = range(5)
PLANNER_GREEDY, PLANNER_EXHAUSTIVE, PLANNER_LEARNED, PLANNER_AUTO = range(4)
FLAG_NO_RENORM = 1
FLAG_REUSE = 2
FLAG_NO_FUSE = 4
FLAG_NO_SMALLK = 8
PREC_NAMES = {"fp32": PREC_FP32, "tf32": PREC_TF32, "bf16": PREC_BF16, "bf16x3": PREC_BF16X3, "auto": PREC_AUTO}

# every symbol include/tqc.h declares
EXPORTS = ["tqc_network_create", "tqc_network_upload", "tqc_destroy", "tqc_plan_opts_default", "tqc_plan",
           "tqc_plan_info", "tqc_plan_step", "tqc_plan_describe", "tqc_contract", "tqc_contract_states",
           "tqc_contract_host",
           "tqc_contract_batch", "tqc_plan_profile", "tqc_plan_step_time", "tqc_plan_destroy", "tqc_last_error",
           "tqc_contract_noalloc", "tqc_noalloc_scratch_bytes", "tqc_costmodel_create", "tqc_costmodel_destroy",
           "tqc_costmodel_params", "tqc_costmodel_set_params", "tqc_costmodel_grad", "tqc_costmodel_train",
           "tqc_costmodel_predict", "tqc_costmodel_save", "tqc_costmodel_load", "tqc_plan_features",
           "tqc_plan_candidates", "tqc_batch_status", "tqc_batch_inject_stall", "tqc_step_inject_stall", "tqc_hss_norms", "tqc_hss_select",
           "tqc_batch_tail_threshold", "tqc_batch_launches", "tqc_network_select", "tqc_cut_opts_default", "tqc_find_cuts", "tqc_plan_cost_report"]
PLAN_FEATURES = 32


class TqcError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"tqc status {status}: {msg}")
        self.status = status


class Subcircuit(ctypes.Structure):
    _fields_ = [("n_out", ctypes.c_int32), ("out_qubits", ctypes.c_void_p),
                ("n_cut", ctypes.c_int32), ("cut_ids", ctypes.c_void_p),
                ("cut_role", ctypes.c_void_p), ("dtype", ctypes.c_int32), ("data", ctypes.c_void_p)]


class PlanOpts(ctypes.Structure):
    _fields_ = [("use_free_mask", ctypes.c_int32), ("free_mask_lo", ctypes.c_uint64),
                ("free_mask_hi", ctypes.c_uint64), ("fixed_bits", ctypes.c_void_p),
                ("precision", ctypes.c_int32), ("planner", ctypes.c_int32),
                ("mem_budget_bytes", ctypes.c_uint64), ("costmodel_path", ctypes.c_char_p),
                ("autotune", ctypes.c_int32), ("n_order", ctypes.c_int32), ("order", ctypes.c_void_p),
                ("n_sliced", ctypes.c_int32), ("sliced_cuts", ctypes.c_void_p), ("flags", ctypes.c_int32)]


_lib = None


def lib():
    """Load libtqc.so (built by ``__graft_entry__.build()``); raises if absent."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"libtqc.so is not built ({LIB_PATH}); run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        vp, i32, u8p = ctypes.c_void_p, ctypes.c_int32, ctypes.c_void_p
        L.tqc_network_create.argtypes = [i32, i32, vp, ctypes.POINTER(vp)]
        L.tqc_network_upload.argtypes = [vp, i32, i32, vp, vp]
        L.tqc_destroy.argtypes = [vp]
        L.tqc_plan_opts_default.argtypes = [ctypes.POINTER(PlanOpts)]
        L.tqc_plan_opts_default.restype = None
        L.tqc_plan.argtypes = [vp, ctypes.POINTER(PlanOpts), ctypes.POINTER(vp)]
        L.tqc_plan_info.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double),
                                    ctypes.POINTER(i32), ctypes.POINTER(i32)]
        L.tqc_plan_step.argtypes = [vp, i32] + [ctypes.POINTER(i32)] * 5
        L.tqc_plan_describe.argtypes = [vp, ctypes.c_char_p, i32]
        L.tqc_plan_describe.restype = i32
        L.tqc_contract.argtypes = [vp, u8p, vp, i32, ctypes.POINTER(ctypes.c_double), vp]
        L.tqc_contract_host.argtypes = [vp, vp, i32, vp, i32, ctypes.POINTER(ctypes.c_double), vp]
        L.tqc_contract_states.argtypes = [vp, vp, ctypes.c_int64, vp, i32, ctypes.POINTER(ctypes.c_double), vp]
        L.tqc_contract_states.restype = ctypes.c_int
        L.tqc_contract_batch.argtypes = [vp, vp, i32, vp]
        L.tqc_plan_destroy.argtypes = [vp]
        L.tqc_plan_profile.argtypes = [vp, i32]
        L.tqc_plan_step_time.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(i32)]
        L.tqc_last_error.restype = ctypes.c_char_p
        L.tqc_contract_noalloc.argtypes = [vp, vp, i32, u8p, vp, i32, vp]
        L.tqc_contract_noalloc.restype = ctypes.c_int
        L.tqc_noalloc_scratch_bytes.argtypes = []
        L.tqc_noalloc_scratch_bytes.restype = ctypes.c_int64
        fp, i32p = ctypes.POINTER(ctypes.c_float), ctypes.POINTER(i32)
        L.tqc_costmodel_create.argtypes = [i32, ctypes.c_uint64, ctypes.POINTER(vp)]
        L.tqc_costmodel_destroy.argtypes = [vp]
        L.tqc_costmodel_params.argtypes = [vp, vp, i32p]
        L.tqc_costmodel_set_params.argtypes = [vp, vp, i32]
        L.tqc_costmodel_grad.argtypes = [vp, vp, vp, i32, vp, fp]
        L.tqc_costmodel_train.argtypes = [vp, vp, vp, i32, i32, i32, ctypes.c_float, ctypes.c_uint64, fp]
        L.tqc_costmodel_predict.argtypes = [vp, vp, i32, vp]
        L.tqc_costmodel_save.argtypes = [vp, ctypes.c_char_p]
        L.tqc_costmodel_load.argtypes = [ctypes.c_char_p, ctypes.POINTER(vp)]
        L.tqc_plan_features.argtypes = [vp, vp, i32]
        L.tqc_plan_candidates.argtypes = [vp, ctypes.POINTER(PlanOpts), i32, vp, i32p]
        L.tqc_batch_status.argtypes = [vp]
        L.tqc_batch_inject_stall.argtypes = [i32]
        L.tqc_batch_tail_threshold.argtypes = [ctypes.c_double]
        L.tqc_batch_tail_threshold.restype = ctypes.c_int
        L.tqc_batch_launches.argtypes = [ctypes.POINTER(ctypes.c_int64), ctypes.POINTER(ctypes.c_int64)]
        L.tqc_batch_launches.restype = ctypes.c_int
        L.tqc_step_inject_stall.argtypes = [i32]
        L.tqc_step_inject_stall.restype = ctypes.c_int
        L.tqc_hss_norms.argtypes = [vp, i32, vp, vp]
        L.tqc_hss_select.argtypes = [vp, ctypes.c_int64, vp, vp, ctypes.c_int64, ctypes.POINTER(ctypes.c_int64)]
        L.tqc_network_select.argtypes = [vp, vp, vp, ctypes.POINTER(vp)]
        L.tqc_cut_opts_default.argtypes = [vp]
        L.tqc_cut_opts_default.restype = None
        L.tqc_find_cuts.argtypes = [i32, i32, vp, vp, vp, vp]
        L.tqc_find_cuts.restype = ctypes.c_int
        L.tqc_plan_cost_report.argtypes = [vp, vp]
        L.tqc_plan_cost_report.restype = ctypes.c_int
        for name in ["tqc_hss_norms", "tqc_hss_select", "tqc_network_select"]:
            getattr(L, name).restype = ctypes.c_int
        for name in ["tqc_batch_status", "tqc_batch_inject_stall", "tqc_costmodel_create", "tqc_costmodel_destroy",
                     "tqc_costmodel_params",
                     "tqc_costmodel_set_params", "tqc_costmodel_grad", "tqc_costmodel_train",
                     "tqc_costmodel_predict", "tqc_costmodel_save", "tqc_costmodel_load", "tqc_plan_features",
                     "tqc_plan_candidates"]:
            getattr(L, name).restype = ctypes.c_int
        for name in ["tqc_network_create", "tqc_network_upload", "tqc_destroy", "tqc_plan", "tqc_plan_info",
                     "tqc_plan_step", "tqc_contract", "tqc_contract_host", "tqc_contract_batch",
                     "tqc_plan_destroy", "tqc_plan_profile", "tqc_plan_step_time"]:
            getattr(L, name).restype = ctypes.c_int
        _lib = L
    return _lib


def _check(st):
    if st != OK:
        raise TqcError(st, lib().tqc_last_error().decode())


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


class Network:
    """A network handle.  ``net`` is any object with ``n_qubits`` and
    ``nodes`` (each with ``out_qubits``, ``cut_ids``, ``cut_role`` and a
    float64/float32 ``data`` array in the row-major [c_0]..[x] layout)."""

    def __init__(self, net, dtype=F64, shape_only=False):
        L = lib()
        self.n_qubits = net.n_qubits
        self.m = len(net.nodes)
        self._keep = []
        subs = (Subcircuit * self.m)()
        npdt = np.float64 if dtype == F64 else np.float32
        for j, nd in enumerate(net.nodes):
            oq = np.ascontiguousarray(nd.out_qubits, dtype=np.int32)
            ci = np.ascontiguousarray(nd.cut_ids, dtype=np.int32)
            cr = np.ascontiguousarray(nd.cut_role, dtype=np.int8)
            data = None if shape_only else np.ascontiguousarray(nd.data, dtype=npdt)
            self._keep += [oq, ci, cr, data]
            subs[j] = Subcircuit(len(oq), oq.ctypes.data if len(oq) else None, len(ci),
                                 ci.ctypes.data if len(ci) else None, cr.ctypes.data if len(cr) else None,
                                 dtype, None if data is None else data.ctypes.data)
        h = ctypes.c_void_p()
        _check(L.tqc_network_create(self.n_qubits, self.m, ctypes.cast(subs, ctypes.c_void_p), ctypes.byref(h)))
        self._keep = None
        self.handle = h
        self.dtype = dtype
        self.plans = []

    @classmethod
    def _wrap(cls, handle, n_qubits, m, dtype):
        self = cls.__new__(cls)
        self.handle, self.n_qubits, self.m, self.dtype, self.plans, self._keep = handle, n_qubits, m, dtype, [], None
        return self

    def hss_norms(self, sub, out, stream=None):
        """L2 norms over the cut assignments of every output state of
        subcircuit ``sub`` into ``out`` (CUDA float64 tensor)."""
        assert out.is_cuda and out.is_contiguous()
        _check(lib().tqc_hss_norms(self.handle, int(sub), ctypes.c_void_p(out.data_ptr()), _stream_ptr(stream)))

    def hss_select(self, s_max):
        """Heavy states: (list of ascending state arrays per subcircuit,
        product of the counts)."""
        counts = np.zeros(self.m, np.int32)
        cap = 1 << 22
        states = np.zeros(cap, np.int32)
        n = ctypes.c_int64()
        _check(lib().tqc_hss_select(self.handle, ctypes.c_int64(int(s_max)), counts.ctypes.data, states.ctypes.data,
                                    ctypes.c_int64(cap), ctypes.byref(n)))
        out, off = [], 0
        for c in counts:
            out.append(states[off:off + c].copy())
            off += c
        return out, n.value

    def select(self, selection):
        """The network restricted to the product of the selected states
        (see tqc_network_select); its outputs are the selection indices."""
        counts = np.ascontiguousarray([len(x) for x in selection], np.int32)
        states = np.ascontiguousarray(np.concatenate([np.asarray(x, np.int64) for x in selection]), np.int32)
        h = ctypes.c_void_p()
        _check(lib().tqc_network_select(self.handle, counts.ctypes.data, states.ctypes.data, ctypes.byref(h)))
        kb = [int(np.ceil(np.log2(c))) if c > 1 else 0 for c in counts]
        return Network._wrap(h, max(1, sum(kb)), self.m, self.dtype)

    def upload(self, sub, host_array, stream=None):
        arr = np.ascontiguousarray(host_array)
        _check(lib().tqc_network_upload(self.handle, sub, self.dtype, arr.ctypes.data, _stream_ptr(stream)))

    def close(self):
        if self.handle:
            for p in list(self.plans):
                p.close()
            _check(lib().tqc_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class CutOpts(ctypes.Structure):
    _fields_ = [("w_max", ctypes.c_int32), ("s_max", ctypes.c_int32), ("k_t", ctypes.c_int32),
                ("k_sweep_max", ctypes.c_int32), ("q_max", ctypes.c_double), ("t_gate", ctypes.c_double),
                ("t_meas", ctypes.c_double), ("shots_log2_min", ctypes.c_int32), ("shots_log2_max", ctypes.c_int32),
                ("n_qpus", ctypes.c_int32), ("cost_free_qubits", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("costmodel_path", ctypes.c_char_p)]


class CutResult(ctypes.Structure):
    _fields_ = [("n_sub", ctypes.c_int32), ("n_cuts", ctypes.c_int32), ("k_t", ctypes.c_int32),
                ("max_width", ctypes.c_int32), ("t_qpu", ctypes.c_double), ("t_classical", ctypes.c_double),
                ("t_total", ctypes.c_double), ("cutqc_mults", ctypes.c_double), ("tensorqc_mults", ctypes.c_double)]


class CostReport(ctypes.Structure):
    _fields_ = [("cutqc_mults_per_state", ctypes.c_double), ("tensorqc_mults_per_state", ctypes.c_double),
                ("ratio", ctypes.c_double), ("plan_mults", ctypes.c_double), ("plan_mults_per_state", ctypes.c_double),
                ("k_max", ctypes.c_int32), ("tn_upper_bound", ctypes.c_double)]


def find_cuts(n_qubits, gates, **opts):
    """Cut finder (tqc_find_cuts): ``gates`` is a list of qubit tuples (one or
    two qubits) in time order; keyword options are tqc_cut_opts fields.
    Returns (per-gate subcircuit ids, result dict)."""
    o = CutOpts()
    lib().tqc_cut_opts_default(ctypes.byref(o))
    for k, v in opts.items():
        if k == "costmodel_path":
            v = v.encode() if v else None
        setattr(o, k, v)
    gq = np.full((max(len(gates), 1), 2), -1, dtype=np.int32)
    for g, qs in enumerate(gates):
        gq[g, :len(qs)] = qs
    part = np.zeros(max(len(gates), 1), dtype=np.int32)
    r = CutResult()
    _check(lib().tqc_find_cuts(n_qubits, len(gates), gq.ctypes.data, ctypes.byref(o), part.ctypes.data,
                               ctypes.byref(r)))
    return part[:len(gates)].tolist(), {f: getattr(r, f) for f, _ in CutResult._fields_}


class Plan:
    def __init__(self, net: Network, precision=PREC_AUTO, planner=PLANNER_AUTO, free_qubits=None,
                 fixed_bits=None, mem_budget=0, order=None, sliced=None, flags=0, autotune=0,
                 costmodel_path=None):
        L = lib()
        o = PlanOpts()
        L.tqc_plan_opts_default(ctypes.byref(o))
        if isinstance(precision, str):
            precision = PREC_NAMES[precision]
        o.precision = precision
        o.planner = planner
        keep = []
        if free_qubits is not None:
            o.use_free_mask = 1
            lo = hi = 0
            for q in free_qubits:
                if q < 64:
                    lo |= 1 << q
                else:
                    hi |= 1 << (q - 64)
            o.free_mask_lo, o.free_mask_hi = lo, hi
            self.free_qubits = sorted(free_qubits)
        else:
            self.free_qubits = list(range(net.n_qubits))
        if fixed_bits is not None:
            fb = np.ascontiguousarray(fixed_bits, dtype=np.uint8)
            keep.append(fb)
            o.fixed_bits = fb.ctypes.data
        o.mem_budget_bytes = int(mem_budget)
        if order is not None:
            od = np.ascontiguousarray(np.array(order, dtype=np.int32).reshape(-1))
            keep.append(od)
            o.n_order = len(od) // 2
            o.order = od.ctypes.data
        if sliced:
            sc = np.ascontiguousarray(sliced, dtype=np.int32)
            keep.append(sc)
            o.n_sliced = len(sc)
            o.sliced_cuts = sc.ctypes.data
        if costmodel_path:
            o.costmodel_path = costmodel_path.encode()
        o.flags = flags
        o.autotune = autotune
        h = ctypes.c_void_p()
        _check(L.tqc_plan(net.handle, ctypes.byref(o), ctypes.byref(h)))
        self.handle = h
        self.net = net
        self.n_qubits = net.n_qubits
        net.plans.append(self)

    @property
    def out_elems(self):
        return 1 << len(self.free_qubits)

    def info(self):
        f, b = ctypes.c_double(), ctypes.c_double()
        ns, nst = ctypes.c_int32(), ctypes.c_int32()
        _check(lib().tqc_plan_info(self.handle, ctypes.byref(f), ctypes.byref(b), ctypes.byref(ns),
                                   ctypes.byref(nst)))
        return {"flops": f.value, "bytes": b.value, "n_slices": ns.value, "n_steps": nst.value}

    def step(self, i):
        vals = [ctypes.c_int32() for _ in range(5)]
        _check(lib().tqc_plan_step(self.handle, i, *[ctypes.byref(v) for v in vals]))
        return dict(zip(["log2_m", "log2_n", "log2_k", "klass", "precision"], [v.value for v in vals]))

    def describe(self):
        n = lib().tqc_plan_describe(self.handle, None, 0)
        buf = ctypes.create_string_buffer(n + 1)
        lib().tqc_plan_describe(self.handle, buf, n + 1)
        return json.loads(buf.value.decode())

    def contract(self, out, fixed_bits=None, want_z=False, stream=None):
        """Reconstruct into ``out`` (a CUDA torch tensor of float32/float64
        with ``out_elems`` elements).  Returns Z when ``want_z``."""
        import torch
        assert out.is_cuda and out.is_contiguous() and out.numel() == self.out_elems
        dt = F64 if out.dtype == torch.float64 else F32
        if out.dtype not in (torch.float32, torch.float64):
            raise TypeError("out must be float32 or float64")
        fb = None
        if fixed_bits is not None:
            fb = np.ascontiguousarray(fixed_bits, dtype=np.uint8)
        z = ctypes.c_double()
        _check(lib().tqc_contract(self.handle, None if fb is None else fb.ctypes.data, out.data_ptr(), dt,
                                  ctypes.byref(z) if want_z else None, _stream_ptr(stream)))
        return z.value if want_z else None

    def contract_states(self, states, out, want_z=False, stream=None):
        """P of each state in ``states`` (ints, or a uint64 array; qubit q =
        bit q) into ``out`` (CUDA float32/float64 tensor of len(states)).
        The plan must have no free qubits (``free_qubits=[]``)."""
        import torch
        st = np.ascontiguousarray(np.asarray(states, dtype=np.uint64))
        assert out.is_cuda and out.is_contiguous() and out.numel() == len(st)
        if out.dtype not in (torch.float32, torch.float64):
            raise TypeError("out must be float32 or float64")
        dt = F64 if out.dtype == torch.float64 else F32
        z = ctypes.c_double()
        _check(lib().tqc_contract_states(self.handle, st.ctypes.data if len(st) else None, len(st),
                                         out.data_ptr() if len(st) else None, dt,
                                         ctypes.byref(z) if want_z else None, _stream_ptr(stream)))
        return z.value if want_z else None

    def contract_host(self, host_tensors, host_out, in_dtype=F64, stream=None):
        """End-to-end: host tensors in (None = unchanged), host results out."""
        arr = (ctypes.c_void_p * self.net.m)()
        keep = []
        for j, t in enumerate(host_tensors or [None] * self.net.m):
            if t is not None:
                keep.append(t)
                arr[j] = t.ctypes.data if isinstance(t, np.ndarray) else t.data_ptr()
        dt = F64 if host_out.dtype in (np.float64,) or str(host_out.dtype) == "torch.float64" else F32
        optr = host_out.ctypes.data if isinstance(host_out, np.ndarray) else host_out.data_ptr()
        z = ctypes.c_double()
        _check(lib().tqc_contract_host(self.handle, ctypes.cast(arr, ctypes.c_void_p) if host_tensors else None,
                                       in_dtype, optr, dt, ctypes.byref(z), _stream_ptr(stream)))
        return z.value

    def contract_noalloc(self, d_tensors, out, in_dtype=F64, fixed_bits=None, stream=None):
        """Allocation-free form: ``d_tensors`` are the caller's device tensors
        (one per subcircuit), every intermediate lives in the library's fixed
        scratch array (see tqc_contract_noalloc in include/tqc.h)."""
        ptrs = (ctypes.c_void_p * len(d_tensors))(*[t.data_ptr() for t in d_tensors])
        fb = None if fixed_bits is None else np.ascontiguousarray(fixed_bits, dtype=np.uint8)
        import torch
        dt = F64 if out.dtype == torch.float64 else F32
        _check(lib().tqc_contract_noalloc(self.handle, ctypes.cast(ptrs, ctypes.c_void_p), in_dtype,
                                          None if fb is None else fb.ctypes.data, out.data_ptr(), dt,
                                          _stream_ptr(stream)))

    def cost_report(self):
        """Multiplications of this plan against the brute-force
        reconstruction (tqc_plan_cost_report)."""
        r = CostReport()
        _check(lib().tqc_plan_cost_report(self.handle, ctypes.byref(r)))
        return {f: getattr(r, f) for f, _ in CostReport._fields_}

    def features(self):
        """The plan's TQC_PLAN_FEATURES cost-model features (float32)."""
        f = np.zeros(PLAN_FEATURES, np.float32)
        _check(lib().tqc_plan_features(self.handle, f.ctypes.data, PLAN_FEATURES))
        return f

    def profile(self, enable=True):
        _check(lib().tqc_plan_profile(self.handle, int(enable)))

    def step_time(self, i):
        """(mean ms, launches) of step i over the profiled contracts."""
        ms, n = ctypes.c_double(), ctypes.c_int32()
        _check(lib().tqc_plan_step_time(self.handle, i, ctypes.byref(ms), ctypes.byref(n)))
        return ms.value, n.value

    def close(self):
        if self.handle:
            _check(lib().tqc_plan_destroy(self.handle))
            self.handle = None
            if self in self.net.plans:
                self.net.plans.remove(self)

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def plan_candidates(net: Network, max_n=24, precision=PREC_AUTO, free_qubits=None):
    """Candidate contraction orders (lists of (a, b) pairs) of a network."""
    o = PlanOpts()
    lib().tqc_plan_opts_default(ctypes.byref(o))
    o.precision = PREC_NAMES[precision] if isinstance(precision, str) else precision
    if free_qubits is not None:
        o.use_free_mask = 1
        o.free_mask_lo = sum(1 << q for q in free_qubits if q < 64)
        o.free_mask_hi = sum(1 << (q - 64) for q in free_qubits if q >= 64)
    per = 2 * (net.m - 1)
    buf = np.zeros(max(1, max_n * per), np.int32)
    n = ctypes.c_int32()
    _check(lib().tqc_plan_candidates(net.handle, ctypes.byref(o), max_n, buf.ctypes.data, ctypes.byref(n)))
    return [buf[i * per:(i + 1) * per].reshape(-1, 2).tolist() for i in range(n.value)]


class CostModel:
    """The learned cost model (include/tqc.h, tqc_costmodel_*)."""

    def __init__(self, n_features=PLAN_FEATURES, seed=0, _handle=None):
        if _handle is not None:
            self.handle = _handle
        else:
            h = ctypes.c_void_p()
            _check(lib().tqc_costmodel_create(n_features, seed, ctypes.byref(h)))
            self.handle = h
        self.n_features = n_features

    @classmethod
    def load(cls, path):
        h = ctypes.c_void_p()
        _check(lib().tqc_costmodel_load(path.encode(), ctypes.byref(h)))
        return cls(_handle=h)

    def save(self, path):
        _check(lib().tqc_costmodel_save(self.handle, path.encode()))

    def params(self):
        n = ctypes.c_int32()
        _check(lib().tqc_costmodel_params(self.handle, None, ctypes.byref(n)))
        out = np.zeros(n.value, np.float32)
        _check(lib().tqc_costmodel_params(self.handle, out.ctypes.data, ctypes.byref(n)))
        return out

    def set_params(self, theta):
        th = np.ascontiguousarray(theta, np.float32)
        _check(lib().tqc_costmodel_set_params(self.handle, th.ctypes.data, len(th)))

    def grad(self, X, t):
        X = np.ascontiguousarray(X, np.float32)
        t = np.ascontiguousarray(t, np.float32)
        g = np.zeros(len(self.params()), np.float32)
        loss = ctypes.c_float()
        _check(lib().tqc_costmodel_grad(self.handle, X.ctypes.data, t.ctypes.data, len(t), g.ctypes.data,
                                        ctypes.byref(loss)))
        return loss.value, g

    def train(self, X, logt, epochs=200, batch=64, lr=1e-3, seed=0):
        X = np.ascontiguousarray(X, np.float32)
        y = np.ascontiguousarray(logt, np.float32)
        loss = ctypes.c_float()
        _check(lib().tqc_costmodel_train(self.handle, X.ctypes.data, y.ctypes.data, len(y), epochs, batch, lr, seed,
                                         ctypes.byref(loss)))
        return loss.value

    def predict(self, X):
        X = np.ascontiguousarray(X, np.float32)
        out = np.zeros(len(X), np.float32)
        _check(lib().tqc_costmodel_predict(self.handle, X.ctypes.data, len(X), out.ctypes.data))
        return out

    def close(self):
        if self.handle:
            _check(lib().tqc_costmodel_destroy(self.handle))
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def contract_batch(plans, outs, stream=None):
    n = len(plans)
    hp = (ctypes.c_void_p * n)(*[p.handle.value for p in plans])
    ho = (ctypes.c_void_p * n)(*[o.data_ptr() for o in outs])
    _check(lib().tqc_contract_batch(ctypes.cast(hp, ctypes.c_void_p), ctypes.cast(ho, ctypes.c_void_p), n,
                                    _stream_ptr(stream)))


def batch_status(stream=None):
    """Synchronise and raise TqcError(ERR_TIMEOUT) if the last batched
    launch had a bounded wait give up."""
    _check(lib().tqc_batch_status(_stream_ptr(stream)))


def batch_tail_threshold(seconds: float):
    """Predicted step time from which a plan's steps run as their own
    launches after the persistent kernel of contract_batch (0 = every step,
    float("inf") = none)."""
    _check(lib().tqc_batch_tail_threshold(min(float(seconds), 1e30)))


def batch_launches():
    """(kernel launches per contract_batch call, steps run after the
    persistent kernel) for the last batch list."""
    n, t = ctypes.c_int64(), ctypes.c_int64()
    _check(lib().tqc_batch_launches(ctypes.byref(n), ctypes.byref(t)))
    return n.value, t.value


def batch_inject_stall(enable: bool):
    """Fault-injection hook: batched launches carry an item whose wait can never be met."""
    _check(lib().tqc_batch_inject_stall(int(enable)))


def step_inject_stall(enable: bool):
    """Fault-injection hook: tensor-core step launches whose first CTA never
    fills its first stage, so a bounded wait gives up (see tqc_step_inject_stall)."""
    _check(lib().tqc_step_inject_stall(int(enable)))
