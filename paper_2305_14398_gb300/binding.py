"""ctypes binding of libtqs.so (include/tqs.h): argument marshalling only.

Every function has the C entry point's name and calls it once.  Device
buffers are torch CUDA tensors (their data_ptr() is passed); streams default
to torch's current stream.  All computation happens in the library's
kernels: if libtqs.so is missing this module raises instead of falling back.
"""
from __future__ import annotations

import ctypes
import os
import re
from typing import Iterable, List, Optional, Sequence, Tuple

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.environ.get("TQS_LIB") or os.path.join(HERE, "libtqs.so")
HEADER = os.path.join(os.path.dirname(HERE), "include", "tqs.h")

GATE_IDS = {"h": 0, "x": 1, "y": 2, "z": 3, "s": 4, "t": 5, "r": 6, "rx": 7, "ry": 8, "rz": 9,
            "u3": 10, "cx": 11, "cnot": 11, "cz": 12, "cp": 13, "cu": 14, "swap": 15,
            "measure": 16, "reset": 17}
TWO_QUBIT_IDS = {11, 12, 13, 14, 15}

PREC_FP32_SIMT = 0
PREC_TC_BF16X3 = 1
PREC_TC_TF32X3 = 2

STATUS = ["TQS_OK", "TQS_ERR_ARG", "TQS_ERR_QUBIT_RANGE", "TQS_ERR_QUBIT_DUP",
          "TQS_ERR_TOO_MANY_QUBITS", "TQS_ERR_NOMEM", "TQS_ERR_BUDGET", "TQS_ERR_CUDA",
          "TQS_ERR_TIMEOUT", "TQS_ERR_STATE", "TQS_ERR_UNSUPPORTED"]


class TqsError(RuntimeError):
    def __init__(self, status: int, message: str):
        name = STATUS[status] if 0 <= status < len(STATUS) else str(status)
        super().__init__(f"{name}: {message}")
        self.status = status
        self.name = name


_lib = None

_vp = ctypes.c_void_p
_i = ctypes.c_int
_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_pi = ctypes.POINTER(ctypes.c_int)
_pd = ctypes.POINTER(ctypes.c_double)

_SIGS = {
    "tqs_circuit_create": (_i, [_i, ctypes.POINTER(_vp)]),
    "tqs_circuit_destroy": (_i, [_vp]),
    "tqs_add_gate": (_i, [_vp, _i, _pi, _i, _pd, _i]),
    "tqs_register_unitary": (_i, [ctypes.c_char_p, _i, _pd]),
    "tqs_add_custom": (_i, [_vp, ctypes.c_char_p, _pi, _i]),
    "tqs_circuit_info": (_i, [_vp, _pi, _pi, _pi]),
    "tqs_circuit_steps": (_i, [_vp, _pi]),
    "tqs_circuit_program": (_i, [_vp, _pi, _pi, _vp, _vp, _vp, ctypes.POINTER(ctypes.c_float),
                                 _pi]),
    "tqs_simulate": (_i, [_vp, _vp, _vp, _vp, _vp, _vp]),
    "tqs_simulate_plain": (_i, [_vp, _vp, _vp, _vp]),
    "tqs_simulate_fsv": (_i, [_vp, _vp, _vp]),
    "tqs_fsv_passes": (_i, [_vp, _pi, _pi]),
    "tqs_simulate_measured": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp]),
    "tqs_materialize_step": (_i, [_vp, _i, _vp, _vp]),
    "tqs_circuit_unitary": (_i, [_vp, _i, _vp, _vp]),
    "tqs_circuit_unitary_cols": (_i, [_vp, _i, _i, _i, _vp, _i64, _vp]),
    "tqs_measure_fp32_peak": (_i, [_i, _pd, _pd, _vp]),
    "tqs_probabilities": (_i, [_vp, _i, _vp, _vp, _vp]),
    "tqs_marginal_zero": (_i, [_vp, _i, _u64, _vp, _vp]),
    "tqs_probabilities_noalloc": (_i, [_vp, _i, _vp, _vp, _vp]),
    "tqs_sample": (_i, [_vp, _i, _i64, _vp, _vp, _vp]),
    "tqs_simulate_and_collapse": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "tqs_batch_sample": (_i, [_vp, _vp, _i, _vp, _vp, _vp]),
    "tqs_batch_create": (_i, [ctypes.POINTER(_vp), _i, ctypes.POINTER(_vp)]),
    "tqs_batch_create_packed": (_i, [_i, _vp, _vp, _vp, _vp, _vp, ctypes.POINTER(_vp)]),
    "tqs_batch_info": (_i, [_vp, _pi, ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                            ctypes.POINTER(_i64), _vp]),
    "tqs_batch_run": (_i, [_vp, _vp, _vp, _vp, _i, _vp]),
    "tqs_batch_run_host": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "tqs_batch_instructions": (_i, [_vp, _vp]),
    "tqs_batch_launch_info": (_i, [_vp, _i, _pi, _pi, _pi, _pi]),
    "tqs_batch_run_measured": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, _i, _vp]),
    "tqs_batch_destroy": (_i, [_vp]),
    "tqs_server_create": (_i, [ctypes.c_size_t, _i, _i, ctypes.POINTER(_vp)]),
    "tqs_server_submit_packed": (_i, [_vp, _i64, _i, _i, _vp, _vp, _vp]),
    "tqs_server_poll": (_i, [_vp, _vp, _i, _pi]),
    "tqs_server_take": (_i, [_vp, _i64, _vp, _vp]),
    "tqs_server_stats": (_i, [_vp, ctypes.POINTER(_i64), ctypes.POINTER(_i64),
                              ctypes.POINTER(_i64), ctypes.POINTER(_i64), ctypes.POINTER(_i64)]),
    "tqs_server_destroy": (_i, [_vp]),
    "tqs_set_option": (_i, [_i, _i, _i64]),
    "tqs_set_allocator": (_i, [_vp, _vp, _vp]),
    "tqs_check_violations": (_i, [_vp, _i]),
    "tqs_server_cancel": (_i, [_vp, _i64]),
    "tqs_get_option": (_i, [_i, _i, ctypes.POINTER(_i64)]),
    "tqs_selftest_wait_timeout": (_i, [_i64, _vp]),
    "tqs_last_error": (ctypes.c_char_p, []),
    "tqs_status_string": (ctypes.c_char_p, [_i]),
    "tqs_launch_count": (_i64, []),
}


def lib():
    """Load libtqs.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2305_14398_gb300.build`")
        L = ctypes.CDLL(LIB_PATH)
        for name, (res, args) in _SIGS.items():
            if hasattr(L, name):
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
        _lib = L
    return _lib


def header_functions() -> List[str]:
    """Names of the functions include/tqs.h declares."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(tqs_[a-z0-9_]+)\s*\(", txt)))


def _check(status: int):
    if status != 0:
        msg = lib().tqs_last_error().decode(errors="replace")
        raise TqsError(status, msg)


def _ptr(t) -> Optional[int]:
    if t is None:
        return None
    return t.data_ptr()


def _stream(stream) -> Optional[int]:
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


# ----------------------------------------------------------------- circuit

def tqs_circuit_create(n_qubits: int) -> int:
    h = _vp()
    _check(lib().tqs_circuit_create(int(n_qubits), ctypes.byref(h)))
    return h.value


def tqs_circuit_destroy(c: int) -> None:
    _check(lib().tqs_circuit_destroy(c))


def tqs_add_gate(c: int, gate, qubits: Sequence[int], params: Sequence[float] = ()) -> None:
    gid = GATE_IDS[gate] if isinstance(gate, str) else int(gate)
    qs = (ctypes.c_int * len(qubits))(*[int(q) for q in qubits])
    ps = (ctypes.c_double * max(1, len(params)))(*[float(p) for p in params])
    _check(lib().tqs_add_gate(c, gid, qs, len(qubits), ps, len(params)))


def tqs_register_unitary(name: str, m) -> None:
    """Register a 2^k x 2^k unitary (complex array) under `name`."""
    m = np.asarray(m, dtype=np.complex128)
    k = int(m.shape[0]).bit_length() - 1
    flat = np.empty(2 * m.size, dtype=np.float64)
    flat[0::2] = m.real.reshape(-1)
    flat[1::2] = m.imag.reshape(-1)
    arr = (ctypes.c_double * flat.size)(*flat.tolist())
    _check(lib().tqs_register_unitary(name.encode(), k, arr))


def tqs_add_custom(c: int, name: str, qubits: Sequence[int]) -> None:
    qs = (ctypes.c_int * len(qubits))(*[int(q) for q in qubits])
    _check(lib().tqs_add_custom(c, name.encode(), qs, len(qubits)))


def _custom_name(qubits, params) -> str:
    import hashlib
    h = hashlib.sha1(np.asarray(params, dtype=np.float64).tobytes()).hexdigest()[:20]
    return f"_m{len(qubits)}_{h}"


def tqs_circuit_info(c: int) -> Tuple[int, int, int]:
    n, g, s = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    _check(lib().tqs_circuit_info(c, ctypes.byref(n), ctypes.byref(g), ctypes.byref(s)))
    return n.value, g.value, s.value


def tqs_circuit_steps(c: int) -> List[int]:
    _, g, _ = tqs_circuit_info(c)
    arr = (ctypes.c_int * max(1, g))()
    _check(lib().tqs_circuit_steps(c, arr))
    return list(arr[:g])


PASS_DTYPE = np.dtype([("L", np.uint8, 4), ("op_begin", np.uint32), ("op_count", np.uint32),
                       ("scale", np.float32)])
OP_DTYPE = np.dtype([("code", np.uint8), ("t", np.uint8), ("c", np.uint8), ("tbit", np.uint8),
                     ("d0one", np.uint8), ("fbit", np.uint8), ("act", np.uint16),
                     ("hc", np.complex64), ("m", np.complex64, 4), ("lo", np.complex64, 4)])


def tqs_circuit_program(c: int):
    """(passes, ops, out_map, out_scale, gen_index) of the compiled fused
    program; out_map: 17 uint16, the columns of the output map and its
    offset (see include/tqs.h)."""
    npass, nops = ctypes.c_int(), ctypes.c_int()
    _check(lib().tqs_circuit_program(c, ctypes.byref(npass), ctypes.byref(nops), None, None, None,
                                     None, None))
    passes = np.zeros(npass.value, dtype=PASS_DTYPE)
    ops = np.zeros(nops.value, dtype=OP_DTYPE)
    pos = np.zeros(17, dtype=np.uint16)
    osc = ctypes.c_float()
    gen = ctypes.c_int()
    _check(lib().tqs_circuit_program(c, None, None, passes.ctypes.data, ops.ctypes.data,
                                     pos.ctypes.data, ctypes.byref(osc), ctypes.byref(gen)))
    return passes, ops, pos, float(osc.value), gen.value


def circuit_from_ops(n: int, ops: Iterable) -> int:
    """tqs_circuit_create + one tqs_add_gate per (name, qubits, params)."""
    c = tqs_circuit_create(n)
    try:
        for name, qs, ps in ops:
            if name == "unitary":
                # ("unitary", qubits, params): params = the 2^k x 2^k matrix,
                # row-major, interleaved (re, im)
                v = np.asarray(ps, dtype=np.float64)
                d = 1 << len(qs)
                key = _custom_name(qs, v)
                tqs_register_unitary(key, (v[0::2] + 1j * v[1::2]).reshape(d, d))
                tqs_add_custom(c, key, qs)
            else:
                tqs_add_gate(c, name, qs, ps)
    except Exception:
        tqs_circuit_destroy(c)
        raise
    return c


# ---------------------------------------------------------------- simulate

def tqs_simulate(c: int, out, init=None, probs=None, norm=None, stream=None) -> None:
    _check(lib().tqs_simulate(c, _ptr(init), _ptr(out), _ptr(probs), _ptr(norm), _stream(stream)))


def tqs_simulate_measured(c: int, out, u=None, outcomes=None, init=None, probs=None, norm=None,
                          stream=None) -> None:
    """Circuits with measure / reset instructions: u (float64, one per
    instruction), outcomes (int32, one per instruction)."""
    _check(lib().tqs_simulate_measured(c, _ptr(init), _ptr(out), _ptr(probs), _ptr(norm), _ptr(u),
                                       _ptr(outcomes), _stream(stream)))


def tqs_simulate_fsv(c: int, state, stream=None) -> None:
    """Full-state-vector backend: the circuit applied to `state` in place."""
    _check(lib().tqs_simulate_fsv(c, _ptr(state), _stream(stream)))


def tqs_fsv_passes(c: int) -> Tuple[int, int]:
    """(passes, tile bits) of the circuit's full-state-vector program."""
    p, t = ctypes.c_int(), ctypes.c_int()
    _check(lib().tqs_fsv_passes(c, ctypes.byref(p), ctypes.byref(t)))
    return p.value, t.value


def tqs_simulate_plain(c: int, out, init=None, stream=None) -> None:
    _check(lib().tqs_simulate_plain(c, _ptr(init), _ptr(out), _stream(stream)))


def tqs_materialize_step(c: int, step: int, S, stream=None) -> None:
    _check(lib().tqs_materialize_step(c, int(step), _ptr(S), _stream(stream)))


def tqs_circuit_unitary(c: int, prec: int, U, stream=None) -> None:
    _check(lib().tqs_circuit_unitary(c, int(prec), _ptr(U), _stream(stream)))


def tqs_circuit_unitary_cols(c: int, prec: int, col0: int, ncols: int, U, ldu: Optional[int] = None,
                             stream=None) -> None:
    """Columns [col0, col0 + ncols) of the circuit unitary into U (a 2^n x ldu
    row-major view; ldu defaults to ncols, a compact block)."""
    _check(lib().tqs_circuit_unitary_cols(c, int(prec), int(col0), int(ncols), _ptr(U),
                                          int(ncols if ldu is None else ldu), _stream(stream)))


def tqs_probabilities(state, n: int, probs=None, total=None, stream=None) -> None:
    _check(lib().tqs_probabilities(_ptr(state), int(n), _ptr(probs), _ptr(total), _stream(stream)))


def tqs_probabilities_noalloc(state, n: int, probs=None, total=None, stream=None) -> None:
    _check(lib().tqs_probabilities_noalloc(_ptr(state), int(n), _ptr(probs), _ptr(total),
                                           _stream(stream)))


def tqs_marginal_zero(state, n: int, mask: int, out, stream=None) -> None:
    _check(lib().tqs_marginal_zero(_ptr(state), int(n), int(mask), _ptr(out), _stream(stream)))


# ---------------------------------------------------------------- collapse

def tqs_sample(probs, n: int, shots: int, u, out, stream=None) -> None:
    """Inverse-CDF samples: out[k] (int64) from uniform u[k] (float64)."""
    _check(lib().tqs_sample(_ptr(probs), int(n), int(shots), _ptr(u), _ptr(out), _stream(stream)))


def tqs_simulate_and_collapse(c: int, u, index, state=None, stream=None) -> None:
    """simulateAndCollapse: index[0] (int64) drawn with u[0]; state <- |index>."""
    _check(lib().tqs_simulate_and_collapse(c, _ptr(u), _ptr(index), _ptr(state),
                                           _stream(stream)))


def tqs_batch_sample(b: int, probs, shots: int, u, out, stream=None) -> None:
    """`shots` samples per circuit of a batch (layout circuit-major)."""
    _check(lib().tqs_batch_sample(b, _ptr(probs), int(shots), _ptr(u), _ptr(out),
                                  _stream(stream)))


# ------------------------------------------------------------------- batch

def tqs_batch_create(circuits: Sequence[int]) -> int:
    arr = (_vp * len(circuits))(*circuits)
    h = _vp()
    _check(lib().tqs_batch_create(arr, len(circuits), ctypes.byref(h)))
    return h.value


def pack_ops(circuits: Sequence[Tuple[int, Sequence]]):
    """Host arrays of tqs_batch_create_packed from [(n, ops), ...]."""
    count = len(circuits)
    nq = np.empty(count, dtype=np.int32)
    off = np.zeros(count + 1, dtype=np.int64)
    for i, (n, ops) in enumerate(circuits):
        nq[i] = n
        off[i + 1] = off[i] + len(ops)
    G = int(off[-1])
    kind = np.empty(max(G, 1), dtype=np.int32)
    qub = np.zeros((max(G, 1), 2), dtype=np.int32)
    par = np.zeros((max(G, 1), 8), dtype=np.float64)
    k = 0
    for n, ops in circuits:
        for name, qs, ps in ops:
            kind[k] = GATE_IDS[name]
            qub[k, :len(qs)] = qs
            par[k, :len(ps)] = ps
            k += 1
    return nq, off, kind, qub, par


def tqs_batch_create_packed(nq, off, kind, qub, par) -> int:
    nq = np.ascontiguousarray(nq, dtype=np.int32)
    off = np.ascontiguousarray(off, dtype=np.int64)
    kind = np.ascontiguousarray(kind, dtype=np.int32)
    qub = np.ascontiguousarray(qub, dtype=np.int32)
    par = np.ascontiguousarray(par, dtype=np.float64)
    h = _vp()
    _check(lib().tqs_batch_create_packed(len(nq), nq.ctypes.data, off.ctypes.data, kind.ctypes.data,
                                         qub.ctypes.data, par.ctypes.data, ctypes.byref(h)))
    return h.value


def tqs_batch_info(b: int, extra: bool = False):
    """(count, total_amps, offsets) or, with extra, also (total_steps, program_bytes)."""
    count, total, steps, pbytes = ctypes.c_int(), _i64(), _i64(), _i64()
    _check(lib().tqs_batch_info(b, ctypes.byref(count), ctypes.byref(total), ctypes.byref(steps),
                                ctypes.byref(pbytes), None))
    offs = np.empty(count.value + 1, dtype=np.int64)
    _check(lib().tqs_batch_info(b, None, None, None, None, offs.ctypes.data))
    if extra:
        return count.value, total.value, offs, steps.value, pbytes.value
    return count.value, total.value, offs


def tqs_batch_run(b: int, states, probs=None, norms=None, use_graph: bool = True, stream=None) -> None:
    _check(lib().tqs_batch_run(b, _ptr(states), _ptr(probs), _ptr(norms), int(bool(use_graph)),
                               _stream(stream)))


def tqs_batch_instructions(b: int) -> np.ndarray:
    """Instruction offsets (count + 1 int64) of a batch."""
    count = ctypes.c_int()
    _check(lib().tqs_batch_info(b, ctypes.byref(count), None, None, None, None))
    off = np.empty(count.value + 1, dtype=np.int64)
    _check(lib().tqs_batch_instructions(b, off.ctypes.data))
    return off


def tqs_batch_launch_info(b: int, size_class: int):
    """{"jobs", "grid", "threads", "teams"} of one size class's last launch."""
    v = [ctypes.c_int() for _ in range(4)]
    _check(lib().tqs_batch_launch_info(b, size_class, *[ctypes.byref(x) for x in v]))
    return dict(zip(("jobs", "grid", "threads", "teams"), (x.value for x in v)))


def tqs_batch_run_measured(b: int, states, u, outcomes=None, probs=None, norms=None,
                           use_graph: bool = True, stream=None) -> None:
    _check(lib().tqs_batch_run_measured(b, _ptr(states), _ptr(probs), _ptr(norms), _ptr(u),
                                        _ptr(outcomes), int(bool(use_graph)), _stream(stream)))


def tqs_batch_run_host(b: int, h_states=None, h_probs=None, h_norms=None, stream=None) -> None:
    """Host buffers: torch CPU tensors (pinned or not) or numpy arrays."""
    def hp(x):
        if x is None:
            return None
        if isinstance(x, np.ndarray):
            return x.ctypes.data
        return x.data_ptr()
    _check(lib().tqs_batch_run_host(b, hp(h_states), hp(h_probs), hp(h_norms), _stream(stream)))


def tqs_batch_destroy(b: int) -> None:
    _check(lib().tqs_batch_destroy(b))


def tqs_measure_fp32_peak(iters: int = 20000, stream=None):
    """(TFLOP/s, ms) of the FP32 FMA microkernel."""
    t, ms = ctypes.c_double(), ctypes.c_double()
    _check(lib().tqs_measure_fp32_peak(int(iters), ctypes.byref(t), ctypes.byref(ms), _stream(stream)))
    return t.value, ms.value


def tqs_launch_count() -> int:
    return int(lib().tqs_launch_count())


def tqs_check_violations(reset: bool = False) -> int:
    """Out-of-range accesses the bounds-checked library (libtqs_checked.so)
    has recorded; always 0 for the normal build."""
    v = ctypes.c_uint32()
    _check(lib().tqs_check_violations(ctypes.byref(v), 1 if reset else 0))
    return int(v.value)


def tqs_last_error() -> str:
    return lib().tqs_last_error().decode(errors="replace")


def tqs_status_string(s: int) -> str:
    return lib().tqs_status_string(int(s)).decode()


# ------------------------------------------------------------------ server

def tqs_server_create(hbm_budget_bytes: int, max_inflight: int = 4, max_batch: int = 256) -> int:
    h = _vp()
    _check(lib().tqs_server_create(int(hbm_budget_bytes), int(max_inflight), int(max_batch),
                                   ctypes.byref(h)))
    return h.value


def pack_request(ops):
    """(kind, qubits, params) host arrays of one request."""
    g = max(len(ops), 1)
    kind = np.zeros(g, dtype=np.int32)
    qub = np.zeros((g, 2), dtype=np.int32)
    par = np.zeros((g, 8), dtype=np.float64)
    for k, (name, qs, ps) in enumerate(ops):
        kind[k] = GATE_IDS[name]
        qub[k, :len(qs)] = qs
        par[k, :len(ps)] = ps
    return kind, qub, par, len(ops)


def tqs_server_submit_packed(sv: int, tag: int, n_qubits: int, packed) -> None:
    kind, qub, par, n_gates = packed
    _check(lib().tqs_server_submit_packed(sv, int(tag), int(n_qubits), int(n_gates),
                                          kind.ctypes.data, qub.ctypes.data, par.ctypes.data))


def tqs_server_poll(sv: int, max_done: int = 4096) -> np.ndarray:
    buf = np.empty(max_done, dtype=np.int64)
    nd = ctypes.c_int()
    _check(lib().tqs_server_poll(sv, buf.ctypes.data, int(max_done), ctypes.byref(nd)))
    return buf[:nd.value].copy()


def tqs_server_take(sv: int, tag: int, n_qubits=None):
    """(state or None, norm) of a finished request."""
    norm = ctypes.c_double()
    if n_qubits is None:
        _check(lib().tqs_server_take(sv, int(tag), None, ctypes.byref(norm)))
        return None, norm.value
    st = np.empty(1 << n_qubits, dtype=np.complex64)
    _check(lib().tqs_server_take(sv, int(tag), st.ctypes.data, ctypes.byref(norm)))
    return st, norm.value


def tqs_server_stats(sv: int) -> dict:
    v = [_i64() for _ in range(5)]
    _check(lib().tqs_server_stats(sv, *[ctypes.byref(x) for x in v]))
    return dict(zip(("queued", "inflight", "done", "bytes_in_use", "peak_bytes"), [x.value for x in v]))


def tqs_server_destroy(sv: int) -> None:
    _check(lib().tqs_server_destroy(sv))


# ----------------------------------------------------------------- options

OPT_WARPS_PER_CTA = 1
OPT_TEAM_WARPS = 2
OPT_FSV_MAX_GATES = 3
OPT_MULTI_CTAS = 4
OPT_HOST_WRITES = 5
OPT_EXACT_PROBS = 6
OPT_CTA_THREADS = 7
OPT_FSV_TILE_Q = 8
OPT_CHAIN_GROUP = 9
OPT_CHAIN_KCHUNK = 10
OPT_CHAIN_PAIR = 11


def tqs_set_option(option: int, key: int, value: int) -> None:
    _check(lib().tqs_set_option(int(option), int(key), int(value)))


def tqs_get_option(option: int, key: int) -> int:
    v = _i64()
    _check(lib().tqs_get_option(int(option), int(key), ctypes.byref(v)))
    return v.value


def tqs_selftest_wait_timeout(wait_cycles: int, stream=None) -> None:
    _check(lib().tqs_selftest_wait_timeout(int(wait_cycles), _stream(stream)))


# --------------------------------------------------------------- allocator

ALLOC_FN = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_size_t, ctypes.c_void_p, ctypes.c_void_p)
FREE_FN = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
_allocator_refs = None  # keeps the ctypes callbacks alive while installed


def tqs_set_allocator(alloc=None, free=None) -> None:
    """Install alloc(bytes, stream) -> device pointer (0 / None on failure) and
    free(ptr, stream) as the library's device allocator; no arguments restore
    cudaMalloc / cudaFree."""
    global _allocator_refs
    if alloc is None:
        _check(lib().tqs_set_allocator(None, None, None))
        _allocator_refs = None
        return
    ca = ALLOC_FN(lambda n, stream, ctx: alloc(int(n), stream or 0) or None)
    cf = FREE_FN(lambda p, stream, ctx: free(int(p), stream or 0))
    _check(lib().tqs_set_allocator(ctypes.cast(ca, _vp), ctypes.cast(cf, _vp), None))
    _allocator_refs = (ca, cf)


def use_torch_allocator(device=None) -> None:
    """Route the library's device scratch through torch's caching allocator."""
    import torch
    dev = torch.cuda.current_device() if device is None else int(device)

    def alloc(n, stream):
        return torch.cuda.caching_allocator_alloc(n, dev, stream if stream else None)

    def free(p, stream):
        torch.cuda.caching_allocator_delete(p)

    tqs_set_allocator(alloc, free)


def tqs_server_cancel(sv: int, tag: int) -> None:
    _check(lib().tqs_server_cancel(sv, int(tag)))
