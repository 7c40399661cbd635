"""Python binding of the sfsim C ABI (include/sfsim.h): argument marshalling
only. Every computation runs in libsfsim.so; if the library is missing the
calls raise instead of falling back to anything else.

Functions carry the C names. Device buffers are torch tensors (torch supplies
device memory and streams only).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libsfsim.so")

SF_OK, SF_EINVAL, SF_ENOMEM, SF_ECUDA, SF_ETIMEOUT, SF_ECANCELLED, SF_EUNSUPPORTED = 0, -1, -2, -3, -4, -5, -6
SF_H, SF_X_HALF, SF_Y_HALF, SF_T, SF_Z, SF_S, SF_CZ, SF_ISWAP, SF_U1, SF_U2 = range(10)
SF_DEC_SCHMIDT, SF_DEC_BLOCK4 = 0, 1
SF_EXEC_BATCHED, SF_EXEC_PLAIN = 0, 1
SF_SEL_RANGE, SF_SEL_FRACTION, SF_SEL_LIST = 0, 1, 2
SF_PREC_F64, SF_PREC_COMPENSATED = 0, 1
SF_PROJ_A, SF_PROJ_ALTERNATE = 0, 1
SF_NOALLOC_SCRATCH_BYTES = 64 << 20

EXPORTED = [
    "sf_circuit_create", "sf_circuit_parse", "sf_circuit_info", "sf_circuit_destroy",
    "sf_plan_opts_default", "sf_plan_create", "sf_plan_info", "sf_plan_stats", "sf_plan_destroy",
    "sf_selection_size", "sf_selection_ids", "sf_amplitudes", "sf_workspace_size",
    "sf_amplitudes_device", "sf_server_create", "sf_server_submit", "sf_server_wait",
    "sf_server_cancel", "sf_server_times", "sf_server_destroy", "sf_plan_profile",
    "sf_plan_profile_read", "sf_amplitudes_device_noalloc", "sf_plan_segment_stats",
    "sf_plan_describe", "sf_frugal_accept_device", "sf_plan_autotune", "sf_overlap_device",
    "sf_plan_cost_terms", "sf_cost_fit", "sf_cost_predict", "sf_server_set_cost_model", "sf_last_error",
    "sf_plan_status", "sf_debug_inject_wait_timeouts", "sf_probabilities", "sf_probabilities_device",
    "sf_workspace_size_batch", "sf_amplitudes_device_batch", "sf_debug_set_wait_flag", "sf_server_stats",
    "sf_plan_drop_resident",
]


class SFError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"sfsim error {code}: {msg}")
        self.code = code


class sf_gate(ctypes.Structure):
    _fields_ = [("cycle", ctypes.c_int32), ("kind", ctypes.c_int32), ("q0", ctypes.c_int32),
                ("q1", ctypes.c_int32), ("m", ctypes.c_double * 32)]


class sf_plan_opts(ctypes.Structure):
    _fields_ = [("side_b_mask", ctypes.c_uint64), ("decomposition", ctypes.c_int32),
                ("select_prefix_bits", ctypes.c_int32), ("tile_bits", ctypes.c_int32),
                ("fuse_bits", ctypes.c_int32), ("exec_mode", ctypes.c_int32),
                ("defer_last_level", ctypes.c_int32), ("hbm_budget_bytes", ctypes.c_int64),
                ("batch_paths", ctypes.c_int32), ("run_bits", ctypes.c_int32),
                ("jit", ctypes.c_int32), ("split_last", ctypes.c_int32), ("fp32x2", ctypes.c_int32),
                ("dense_finals", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("projector_side", ctypes.c_int32), ("tile_buffers", ctypes.c_int32),
                ("cycle_segments", ctypes.c_int32), ("reserved", ctypes.c_int32 * 2)]


class sf_path_sel(ctypes.Structure):
    _fields_ = [("mode", ctypes.c_int32), ("first", ctypes.c_uint64), ("count", ctypes.c_uint64),
                ("fidelity", ctypes.c_double), ("seed", ctypes.c_uint64),
                ("list", ctypes.POINTER(ctypes.c_uint64)), ("n_list", ctypes.c_int64)]


class sf_request(ctypes.Structure):
    _fields_ = [("d_bitstrings", ctypes.c_void_p), ("n", ctypes.c_int64), ("sel", ctypes.POINTER(sf_path_sel)),
                ("d_out_amps", ctypes.c_void_p), ("accumulate", ctypes.c_int32)]


_lib = None


def lib():
    """Load libsfsim.so (built by paper_1807_10749_gb300.build)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise SFError(SF_EUNSUPPORTED, f"{LIB_PATH} is not built; run __graft_entry__.build()")
        L = ctypes.CDLL(LIB_PATH)
        P, i32, i64, u64 = ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_uint64
        PP = ctypes.POINTER(ctypes.c_void_p)
        sig = {
            "sf_circuit_create": (i32, [i32, i32, P, i64, PP]),
            "sf_circuit_parse": (i32, [ctypes.c_char_p, PP]),
            "sf_circuit_info": (i32, [P, P, P, P]),
            "sf_circuit_destroy": (None, [P]),
            "sf_plan_opts_default": (None, [P]),
            "sf_plan_create": (i32, [P, P, PP]),
            "sf_plan_info": (i32, [P, P, P, P, P, P]),
            "sf_plan_stats": (i32, [P, P, P, P, P, P]),
            "sf_plan_destroy": (None, [P]),
            "sf_selection_size": (i32, [P, P, P, P]),
            "sf_selection_ids": (i32, [P, P, P, u64, P]),
            "sf_amplitudes": (i32, [P, P, i64, P, P, P]),
            "sf_workspace_size": (i32, [P, i64, P, P]),
            "sf_amplitudes_device": (i32, [P, P, i64, P, P, i32, P, ctypes.c_size_t, P]),
            "sf_server_create": (i32, [i64, i32, PP]),
            "sf_server_submit": (i32, [P, P, P, i64, P, P]),
            "sf_server_wait": (i32, [P, u64, i32, P]),
            "sf_server_cancel": (i32, [P, u64]),
            "sf_server_times": (i32, [P, u64, P, P]),
            "sf_server_destroy": (None, [P]),
            "sf_plan_profile": (i32, [P, i32]),
            "sf_plan_profile_read": (i32, [P, i32, P, P, P]),
            "sf_amplitudes_device_noalloc": (i32, [P, P, i64, P, P, i32, P]),
            "sf_plan_segment_stats": (i32, [P, i32, i32, P, P, P]),
            "sf_plan_describe": (i32, [P, P, ctypes.c_size_t, P]),
            "sf_frugal_accept_device": (i32, [P, P, i64, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                              P, P, P]),
            "sf_plan_autotune": (i32, [P, P, P, i64, P, i64, P, P, P]),
            "sf_overlap_device": (i32, [P, P, i64, P, P]),
            "sf_plan_cost_terms": (i32, [P, P, i64, P]),
            "sf_cost_fit": (i32, [P, P, i64, P]),
            "sf_cost_predict": (ctypes.c_double, [P, P]),
            "sf_server_set_cost_model": (i32, [P, P, ctypes.c_double]),
            "sf_last_error": (ctypes.c_char_p, []),
            "sf_plan_status": (i32, [P, P]),
            "sf_debug_inject_wait_timeouts": (i32, [i32]),
            "sf_probabilities": (i32, [P, P, i64, P, i32, P, P]),
            "sf_probabilities_device": (i32, [P, i64, ctypes.c_double, P, P]),
            "sf_workspace_size_batch": (i32, [P, P, i32, P]),
            "sf_amplitudes_device_batch": (i32, [P, P, i32, P, ctypes.c_size_t, P]),
            "sf_debug_set_wait_flag": (i32, [P, i32]),
            "sf_server_stats": (i32, [P, P, P, P]),
            "sf_plan_drop_resident": (i32, [P]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _check(rc):
    if rc != SF_OK:
        raise SFError(rc, lib().sf_last_error().decode(errors="replace"))


def _ptr(a):
    return ctypes.c_void_p(a.ctypes.data)


# ------------------------------------------------------------- circuits
def sf_circuit_parse(text: str) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().sf_circuit_parse(text.encode(), ctypes.byref(h)))
    return h


def sf_circuit_create(rows: int, cols: int, gates) -> ctypes.c_void_p:
    arr = (sf_gate * max(1, len(gates)))()
    for i, g in enumerate(gates):
        arr[i] = g
    h = ctypes.c_void_p()
    _check(lib().sf_circuit_create(rows, cols, ctypes.cast(arr, ctypes.c_void_p), len(gates), ctypes.byref(h)))
    return h


def sf_circuit_info(c):
    r, cc, n = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
    _check(lib().sf_circuit_info(c, ctypes.byref(r), ctypes.byref(cc), ctypes.byref(n)))
    return r.value, cc.value, n.value


def sf_circuit_destroy(c):
    lib().sf_circuit_destroy(c)


# ---------------------------------------------------------------- plans
def sf_plan_opts_default(**kw) -> sf_plan_opts:
    o = sf_plan_opts()
    lib().sf_plan_opts_default(ctypes.byref(o))
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def sf_plan_create(circuit, opts: sf_plan_opts | None = None) -> ctypes.c_void_p:
    h = ctypes.c_void_p()
    _check(lib().sf_plan_create(circuit, ctypes.byref(opts) if opts is not None else None, ctypes.byref(h)))
    return h


def sf_plan_info(plan):
    v = [ctypes.c_int() for _ in range(5)]
    _check(lib().sf_plan_info(plan, *[ctypes.byref(x) for x in v]))
    return dict(zip(["n_cross", "path_bits", "m_a", "m_b", "n_levels"], [x.value for x in v]))


def sf_plan_stats(plan):
    v = [ctypes.c_int() for _ in range(5)]
    _check(lib().sf_plan_stats(plan, *[ctypes.byref(x) for x in v]))
    return dict(zip(["passes_a", "passes_b", "stages_a", "stages_b", "deferred"], [x.value for x in v]))


def sf_plan_segment_stats(plan, half, segment):
    """(passes, stages, algorithmic bytes per node) of one segment of one half."""
    a, b, c = ctypes.c_int(), ctypes.c_int(), ctypes.c_double()
    _check(lib().sf_plan_segment_stats(plan, half, segment, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def sf_plan_describe(plan) -> str:
    n = ctypes.c_size_t()
    _check(lib().sf_plan_describe(plan, None, 0, ctypes.byref(n)))
    buf = ctypes.create_string_buffer(n.value + 1)
    _check(lib().sf_plan_describe(plan, buf, n.value + 1, ctypes.byref(n)))
    return buf.value.decode()


def sf_plan_autotune(circuit, base: sf_plan_opts, sel, sample_paths, d_bits):
    """Fastest options for this circuit and request sample, timed on the
    device: returns (sf_plan_opts, its seconds, the base options' seconds)."""
    best = sf_plan_opts()
    t, t0 = ctypes.c_double(), ctypes.c_double()
    _check(lib().sf_plan_autotune(circuit, ctypes.byref(base), ctypes.byref(sel), sample_paths,
                                  ctypes.c_void_p(d_bits.data_ptr()), d_bits.numel(), ctypes.byref(best),
                                  ctypes.byref(t), ctypes.byref(t0)))
    return best, t.value, t0.value


def sf_plan_destroy(plan):
    lib().sf_plan_destroy(plan)


# ------------------------------------------------------------ selection
def selection(mode="range", first=0, count=0, fidelity=1.0, seed=7, ids=None):
    """Build an sf_path_sel. The returned object keeps `ids` alive."""
    s = sf_path_sel()
    s.mode = {"range": SF_SEL_RANGE, "fraction": SF_SEL_FRACTION, "list": SF_SEL_LIST}[mode]
    s.first, s.count, s.fidelity, s.seed = first, count, fidelity, seed
    if ids is not None:
        arr = np.ascontiguousarray(ids, dtype=np.uint64)
        s._keep = arr
        s.list = arr.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))
        s.n_list = len(arr)
    return s


def sf_selection_size(plan, sel):
    n, fa = ctypes.c_uint64(), ctypes.c_double()
    _check(lib().sf_selection_size(plan, ctypes.byref(sel), ctypes.byref(n), ctypes.byref(fa)))
    return n.value, fa.value


def sf_selection_ids(plan, sel, cap=None):
    if cap is None:
        cap, _ = sf_selection_size(plan, sel)
    out = np.zeros(max(1, cap), dtype=np.uint64)
    w = ctypes.c_uint64()
    _check(lib().sf_selection_ids(plan, ctypes.byref(sel), _ptr(out), cap, ctypes.byref(w)))
    return out[:w.value]


# ----------------------------------------------------------- amplitudes
def sf_amplitudes(plan, bitstrings, sel):
    """Host form: returns (complex128 amplitudes, f_actual)."""
    bits = np.ascontiguousarray(bitstrings, dtype=np.uint64)
    out = np.zeros(2 * len(bits), dtype=np.float64)
    fa = ctypes.c_double()
    _check(lib().sf_amplitudes(plan, _ptr(bits), len(bits), ctypes.byref(sel), _ptr(out), ctypes.byref(fa)))
    return out[0::2] + 1j * out[1::2], fa.value


def sf_amplitudes_into(plan, bits_u64, sel, out_f64):
    """Host form into caller buffers (e.g. pinned): bits_u64 a contiguous
    uint64 array, out_f64 a contiguous float64 array of 2n (re, im). Returns
    f_actual."""
    assert bits_u64.dtype == np.uint64 and bits_u64.flags["C_CONTIGUOUS"]
    assert out_f64.dtype == np.float64 and out_f64.flags["C_CONTIGUOUS"] and out_f64.size >= 2 * bits_u64.size
    fa = ctypes.c_double()
    _check(lib().sf_amplitudes(plan, _ptr(bits_u64), bits_u64.size, ctypes.byref(sel), _ptr(out_f64),
                               ctypes.byref(fa)))
    return fa.value


def sf_probabilities(plan, bitstrings, sel, divide_by_f=False):
    """Host form: returns (float64 probabilities |amp|^2 [/ f_actual], f_actual)."""
    bits = np.ascontiguousarray(bitstrings, dtype=np.uint64)
    out = np.zeros(len(bits), dtype=np.float64)
    fa = ctypes.c_double()
    _check(lib().sf_probabilities(plan, _ptr(bits), len(bits), ctypes.byref(sel), 1 if divide_by_f else 0,
                                  _ptr(out), ctypes.byref(fa)))
    return out, fa.value


def sf_probabilities_device(d_amps, d_probs, scale=1.0, stream=None):
    """|amp|^2 * scale of float64 (n, 2) device amplitudes into float64 (n,)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(lib().sf_probabilities_device(ctypes.c_void_p(d_amps.data_ptr()), d_probs.numel(), float(scale),
                                         ctypes.c_void_p(d_probs.data_ptr()), ctypes.c_void_p(stream.cuda_stream)))


def sf_plan_status(plan, stream=None):
    """Waits for the stream; raises SFError(SF_ECUDA) if a kernel wait of this
    plan timed out since the last check (and clears the flag)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(lib().sf_plan_status(plan, ctypes.c_void_p(stream.cuda_stream)))


def sf_debug_inject_wait_timeouts(count):
    """Test hook: the next `count` wait-timeout checks report a timeout."""
    _check(lib().sf_debug_inject_wait_timeouts(count))


def sf_plan_drop_resident(plan):
    """Forget resident nodes and free the host-form device buffers."""
    _check(lib().sf_plan_drop_resident(plan))


def sf_debug_set_wait_flag(plan, value=1):
    """Test hook: write `value` into the plan's device wait-timeout flag."""
    _check(lib().sf_debug_set_wait_flag(plan, value))


def _requests(reqs):
    """reqs: [(d_bits, sel, d_out, accumulate)] -> ctypes array (kept alive by the caller)."""
    arr = (sf_request * max(1, len(reqs)))()
    for i, (d_bits, sel, d_out, acc) in enumerate(reqs):
        arr[i].d_bitstrings = d_bits.data_ptr()
        arr[i].n = d_bits.numel()
        arr[i].sel = ctypes.pointer(sel)
        arr[i].d_out_amps = d_out.data_ptr()
        arr[i].accumulate = 1 if acc else 0
    return arr


def sf_workspace_size_batch(plan, reqs) -> int:
    arr = _requests(reqs)
    b = ctypes.c_size_t()
    _check(lib().sf_workspace_size_batch(plan, arr, len(reqs), ctypes.byref(b)))
    return b.value


def sf_amplitudes_device_batch(plan, reqs, workspace, stream=None):
    """Several requests on one plan in one run: reqs = [(d_bits, sel, d_out,
    accumulate)] of torch device tensors (d_out float64 (n, 2))."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    arr = _requests(reqs)
    _check(lib().sf_amplitudes_device_batch(plan, arr, len(reqs), ctypes.c_void_p(workspace.data_ptr()),
                                            workspace.numel(), ctypes.c_void_p(stream.cuda_stream)))


def sf_workspace_size(plan, n, sel) -> int:
    b = ctypes.c_size_t()
    _check(lib().sf_workspace_size(plan, n, ctypes.byref(sel), ctypes.byref(b)))
    return b.value


def sf_amplitudes_device(plan, d_bits, sel, d_out, workspace, stream=None, accumulate=False):
    """Device form. d_bits: torch uint64/int64 (n,), d_out: torch float64 (n, 2),
    workspace: torch uint8 tensor of sf_workspace_size bytes. Enqueues on
    `stream` (torch.cuda.Stream or None for the current stream)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    n = d_bits.numel()
    _check(lib().sf_amplitudes_device(plan, ctypes.c_void_p(d_bits.data_ptr()), n, ctypes.byref(sel),
                                      ctypes.c_void_p(d_out.data_ptr()), 1 if accumulate else 0,
                                      ctypes.c_void_p(workspace.data_ptr()), workspace.numel(),
                                      ctypes.c_void_p(stream.cuda_stream)))


def sf_amplitudes_device_noalloc(plan, d_bits, sel, d_out, stream=None, accumulate=False):
    """Device form without a workspace argument: its scratch is a fixed array
    inside the library, so the call allocates no device memory (see sfsim.h)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(lib().sf_amplitudes_device_noalloc(plan, ctypes.c_void_p(d_bits.data_ptr()), d_bits.numel(),
                                              ctypes.byref(sel), ctypes.c_void_p(d_out.data_ptr()),
                                              1 if accumulate else 0, ctypes.c_void_p(stream.cuda_stream)))


# --------------------------------------------------------------- server
def sf_server_create(hbm_budget_bytes=0, max_concurrent=4):
    h = ctypes.c_void_p()
    _check(lib().sf_server_create(hbm_budget_bytes, max_concurrent, ctypes.byref(h)))
    return h


def sf_server_submit(server, plan, bitstrings, sel):
    bits = np.ascontiguousarray(bitstrings, dtype=np.uint64)
    t = ctypes.c_uint64()
    _check(lib().sf_server_submit(server, plan, _ptr(bits), len(bits), ctypes.byref(sel), ctypes.byref(t)))
    return t.value


def sf_server_wait(server, ticket, n, timeout_ms=-1):
    out = np.zeros(2 * n, dtype=np.float64)
    _check(lib().sf_server_wait(server, ticket, timeout_ms, _ptr(out)))
    return out[0::2] + 1j * out[1::2]


def sf_server_cancel(server, ticket):
    _check(lib().sf_server_cancel(server, ticket))


def sf_server_times(server, ticket):
    q, t = ctypes.c_double(), ctypes.c_double()
    _check(lib().sf_server_times(server, ticket, ctypes.byref(q), ctypes.byref(t)))
    return q.value, t.value


def sf_server_stats(server):
    """(batches, requests in them, largest batch) run by the server."""
    a, b, c = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
    _check(lib().sf_server_stats(server, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)))
    return a.value, b.value, c.value


def sf_server_destroy(server):
    lib().sf_server_destroy(server)


def sf_plan_profile(plan, enable_timing=True):
    _check(lib().sf_plan_profile(plan, 1 if enable_timing else 0))


def sf_plan_profile_read(plan, kernel):
    """(launches, seconds, algorithmic bytes) of kernel 0 pass, 1 gather, 2 other."""
    n, t, b = ctypes.c_int64(), ctypes.c_double(), ctypes.c_double()
    _check(lib().sf_plan_profile_read(plan, kernel, ctypes.byref(n), ctypes.byref(t), ctypes.byref(b)))
    return n.value, t.value, b.value


def sf_frugal_accept_device(d_amps, d_uniform, n_qubits, mprime, d_accept, d_count, prob_scale=1.0,
                            stream=None):
    """Accept step of frugal rejection sampling on device tensors: d_amps
    float64 (n, 2), d_uniform float64 (n,), d_accept uint8 (n,), d_count int64 (1,)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(lib().sf_frugal_accept_device(ctypes.c_void_p(d_amps.data_ptr()), ctypes.c_void_p(d_uniform.data_ptr()),
                                         d_uniform.numel(), float(2.0 ** n_qubits), float(mprime),
                                         float(prob_scale), ctypes.c_void_p(d_accept.data_ptr()),
                                         ctypes.c_void_p(d_count.data_ptr()), ctypes.c_void_p(stream.cuda_stream)))


def sf_overlap_device(d_a, d_b, d_out, stream=None):
    """<a|b> (re, im), <a|a>, <b|b> and the estimate f_e of two float64 (n, 2)
    device tensors into d_out (5,)."""
    import torch
    if stream is None:
        stream = torch.cuda.current_stream()
    _check(lib().sf_overlap_device(ctypes.c_void_p(d_a.data_ptr()), ctypes.c_void_p(d_b.data_ptr()),
                                   d_a.shape[0], ctypes.c_void_p(d_out.data_ptr()),
                                   ctypes.c_void_p(stream.cuda_stream)))


def fidelity_estimate(out):
    """f_e as sf_overlap_device computed it (the fifth of its outputs)."""
    return float(out[4])


def sf_plan_cost_terms(plan, sel, n_a):
    """The four features (1, t1, t2, t3) of the runtime model for a request."""
    t = (ctypes.c_double * 4)()
    _check(lib().sf_plan_cost_terms(plan, ctypes.byref(sel), n_a, t))
    return np.array(t[:], dtype=np.float64)


def sf_cost_fit(terms, seconds):
    """Fit (C0, C1, C1*C2, C3) >= 0 from an (n, 4) feature array and n times."""
    t = np.ascontiguousarray(terms, dtype=np.float64)
    s = np.ascontiguousarray(seconds, dtype=np.float64)
    c = (ctypes.c_double * 4)()
    _check(lib().sf_cost_fit(_ptr(t), _ptr(s), len(s), c))
    return np.array(c[:], dtype=np.float64)


def sf_cost_predict(terms, coeffs):
    t = np.ascontiguousarray(terms, dtype=np.float64)
    c = np.ascontiguousarray(coeffs, dtype=np.float64)
    return float(lib().sf_cost_predict(_ptr(t), _ptr(c)))


def sf_server_set_cost_model(server, coeffs, max_wait_s=1.0):
    if coeffs is None:
        _check(lib().sf_server_set_cost_model(server, None, max_wait_s))
    else:
        c = np.ascontiguousarray(coeffs, dtype=np.float64)
        _check(lib().sf_server_set_cost_model(server, _ptr(c), max_wait_s))


def sf_last_error() -> str:
    return lib().sf_last_error().decode(errors="replace")


# ----------------------------------------------------------- convenience
class Plan:
    """Circuit text + plan options -> an sfsim plan (owns both handles)."""

    def __init__(self, circuit_text: str, **opts):
        self.circuit = sf_circuit_parse(circuit_text)
        try:
            self.handle = sf_plan_create(self.circuit, sf_plan_opts_default(**opts))
        except Exception:
            sf_circuit_destroy(self.circuit)
            self.circuit = None
            raise
        self.info = sf_plan_info(self.handle)

    def amplitudes(self, bitstrings, sel):
        return sf_amplitudes(self.handle, bitstrings, sel)

    def close(self):
        if getattr(self, "handle", None):
            sf_plan_destroy(self.handle)
            self.handle = None
        if getattr(self, "circuit", None):
            sf_circuit_destroy(self.circuit)
            self.circuit = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
