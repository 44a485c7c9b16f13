"""Host logic of the CUDA path, checked on the CPU.

The library compiles a circuit's steps into passes of 4 thread-local qubit
bits (tqs_circuit_program).  This test replays that program in numpy with the
kernel's semantics (butterflies on local bits, pending per-bit phases, far
controls, SWAP relabeling, final qubit map) and compares the final state with
the FP64 oracle.  It also checks the ASAP step table and the error codes.
No GPU is needed: only host entry points are called.
"""
import numpy as np
import pytest

from measure_cases import safe_uniforms, with_instructions
from oracle import collapse, fsv_route, kron_route
from paper_2305_14398_gb300 import binding as B
from paper_2305_14398_gb300 import workloads as W

OPC_H, OPC_X, OPC_XF, OPC_XL, OPC_ANTI, OPC_DENSE, OPC_CDENSE = 0, 4, 8, 12, 28, 32, 36
OPC_HMASK, OPC_XP = 28, 29
OPC_DLISTM = 57
OPC_DLN, OPC_DLF, OPC_DFL, OPC_DFF, OPC_DLL, OPC_DLIST, OPC_DIAG16, OPC_NOP = 40, 44, 48, 52, 53, 54, 55, 56
BIT_MASK = [0xAAAA, 0xCCCC, 0xF0F0, 0xFF00]


def ins0(x, b):
    return ((x >> b) << (b + 1)) | (x & ((1 << b) - 1))


def replay(n, passes, ops, pos, out_scale=1.0, gen_index=0, uniforms=None, outcomes=None,
           customs=(), on_pass=None):
    """The compiled program in FP64 on the CPU.  on_pass(pi, L, st), if given,
    sees the physical state before pass pi (pi = len(passes), L = None: after
    the last pass, before the output map)."""
    nint = max(n, 4)
    st = np.zeros(1 << nint, dtype=np.complex128)
    st[gen_index] = 1.0
    G = (1 << nint) >> 4
    customs = list(customs)
    for pi, ps in enumerate(passes):
        L = [int(v) for v in ps["L"]]
        if on_pass is not None:
            on_pass(pi, L, st)
        if L[0] == 254:  # custom k-qubit unitary: the next custom matrix, on the
            k = L[1]     # physical bits packed 5 bits each in op_count
            assert pi > 0 and 2 <= k <= 5
            m = customs.pop(0)
            assert m.shape == (1 << k, 1 << k)
            bits = [(int(ps["op_count"]) >> (5 * t)) & 31 for t in range(k)]
            mask = int(np.asarray(ps["scale"], dtype=np.float32).view(np.uint32))
            assert mask == sum(1 << b for b in bits) and len(set(bits)) == k and max(bits) < nint
            idx = np.arange(1 << nint)
            base = idx[(idx & mask) == 0]
            loc = np.array([sum(((j >> t) & 1) << bits[t] for t in range(k)) for j in range(1 << k)])
            grp = base[:, None] + loc[None, :]
            st[grp] = st[grp] @ m.T
            continue
        if L[0] == 255:  # measure / reset instruction on physical bit L[1]
            assert pi > 0 and int(ps["op_count"]) == 0
            idx = np.arange(1 << nint)
            bit = (idx >> L[1]) & 1
            p = np.abs(st) ** 2
            s0, t = float(np.sum(p[bit == 0])), float(np.sum(p))
            k = int(ps["op_begin"])
            b = 0 if uniforms[k] * t < s0 else 1
            outcomes.append((k, b))
            kept = np.where(bit == b, st, 0.0) / np.sqrt((s0 if b == 0 else t - s0) / t)
            if L[2] and b == 1:
                st = np.zeros_like(kept)
                st[idx ^ (1 << L[1])] = kept
            else:
                st = kept
            continue
        assert L == sorted(L) and len(set(L)) == 4 and max(L) < nint
        g = np.arange(G, dtype=np.int64)
        base = g
        for l in L:
            base = ins0(base, l)
        offs = np.array([sum(((j >> k) & 1) << L[k] for k in range(4)) for j in range(16)])
        idx = base[:, None] + offs[None, :]
        a = st[idx].copy()
        pend = np.ones((G, 4), dtype=np.complex128)
        sc = np.ones(G, dtype=np.complex128)
        b0, cnt = int(ps["op_begin"]), int(ps["op_count"])
        prog = ops[b0:b0 + cnt]
        skip = set()  # continuation records
        for k, op in enumerate(prog):
            code = int(op["code"])
            if code == OPC_NOP:  # second record of a 16-entry diagonal / a list
                assert k > 0 and (int(prog[k - 1]["code"]) == OPC_DIAG16 or k in skip)
                continue
            if code == OPC_DLISTM:  # phase lists of several targets over the same bits
                tmask, cnt = int(op["t"]), int(op["c"])
                targets = [t for t in range(5) if (tmask >> t) & 1]
                assert len(targets) >= 2 and 1 <= cnt <= 8 and int(op["fbit"]) == 255
                fb = np.frombuffer(np.array([op["hc"]], dtype=np.complex64).tobytes(), dtype=np.uint8)
                on = [np.ones(G, bool) if fb[e] == 255 else ((base >> int(fb[e])) & 1) == 1
                      for e in range(8)]
                for r, t in enumerate(targets):
                    rec = prog[k + r]
                    if r > 0:
                        assert int(rec["code"]) == OPC_NOP
                        skip.add(k + r)
                    vs = np.concatenate([rec["m"], rec["lo"]]).astype(np.complex128)
                    acc = np.ones(G, dtype=np.complex128)
                    for e in range(8):
                        acc[on[e]] *= vs[e]
                    if t < 4:
                        pend[:, t] *= acc
                    else:
                        sc *= acc
                continue
            if code == OPC_DIAG16:  # entry j multiplies local amplitude j
                assert int(prog[k + 1]["code"]) == OPC_NOP
                d = np.concatenate([op["m"], op["lo"], prog[k + 1]["m"], prog[k + 1]["lo"]]).astype(np.complex128)
                a *= d[None, :]
                continue
            m = op["m"].astype(np.complex128)
            fbit = int(op["fbit"])
            far_on = np.ones(G, bool) if fbit == 255 else ((base >> fbit) & 1) == 1
            if code == OPC_DLIST:  # up to 8 phase factors on one position / the group
                tgt, cnt = int(op["t"]), int(op["c"])
                assert 1 <= cnt <= 8 and 0 <= tgt <= 4 and fbit == 255
                fb = np.frombuffer(np.array([op["hc"]], dtype=np.complex64).tobytes(), dtype=np.uint8)
                vs = np.concatenate([op["m"], op["lo"]]).astype(np.complex128)
                acc = np.ones(G, dtype=np.complex128)
                for e in range(cnt):
                    on = np.ones(G, bool) if fb[e] == 255 else ((base >> int(fb[e])) & 1) == 1
                    acc[on] *= vs[e]
                if tgt < 4:
                    pend[:, tgt] *= acc
                else:
                    sc *= acc
                continue
            if code >= OPC_DLN:
                d0, d1, r = m[0], m[1], m[2]
                if int(op["d0one"]):
                    assert d0 == 1
                if code < OPC_DFL:  # local target, none / far control
                    t = code & 3
                    sc[far_on] *= d0
                    pend[far_on, t] *= r
                elif code < OPC_DFF:  # far target, local control
                    c = code & 3
                    v = np.where(((base >> int(op["tbit"])) & 1) == 1, d1, d0)
                    pend[:, c] *= v
                elif code == OPC_DFF:  # far target, none / far control
                    v = np.where(((base >> int(op["tbit"])) & 1) == 1, d1, d0)
                    sc[far_on] *= v[far_on]
                else:
                    assert code == OPC_DLL
                    t, c = int(op["t"]), int(op["c"])
                    for j in range(16):
                        if (j >> c) & 1:
                            a[:, j] *= d1 if (j >> t) & 1 else d0
                continue
            if code == OPC_HMASK:
                # unscaled Hadamards on the positions of the mask in field t
                hm = int(op["t"])
                assert 2 <= bin(hm).count("1") and hm < 16 and fbit == 255
                for t in range(4):
                    if not (hm >> t) & 1:
                        continue
                    for j in range(16):
                        if (j >> t) & 1:
                            a[:, j] *= pend[:, t]
                    pend[:, t] = 1.0
                    for p in range(8):
                        j0 = ((p >> t) << (t + 1)) | (p & ((1 << t) - 1))
                        j1 = j0 | (1 << t)
                        x0, x1 = a[:, j0].copy(), a[:, j1].copy()
                        a[:, j0], a[:, j1] = x0 + x1, x0 - x1
                continue
            if code == OPC_XP:
                # exchanges on position t where act's bit XOR the far parity is 1
                t, act = int(op["t"]), int(op["act"])
                far = int(np.frombuffer(op["hc"].tobytes()[:4], dtype=np.uint32)[0])
                assert fbit == 255
                par = np.array([bin(int(v) & far).count("1") & 1 for v in base])
                for j in range(16):
                    if (j >> t) & 1:
                        a[:, j] *= pend[:, t]
                pend[:, t] = 1.0
                for p in range(8):
                    j0 = ((p >> t) << (t + 1)) | (p & ((1 << t) - 1))
                    j1 = j0 | (1 << t)
                    on = (((act >> j0) & 1) ^ par) == 1
                    x0, x1 = a[:, j0].copy(), a[:, j1].copy()
                    a[on, j0], a[on, j1] = x1[on], x0[on]
                continue
            act = int(op["act"])
            if code < OPC_X:
                kind, t = "h", code & 3
                m = np.array([1, 1, 1, -1], dtype=np.complex128)
                assert fbit == 255
            elif code < OPC_XF:
                kind, t = "x", code & 3
                assert fbit == 255
            elif code < OPC_XL:
                kind, t = "x", code & 3
            elif code < OPC_ANTI:
                kind, t, cl = "x", (code - OPC_XL) >> 2, (code - OPC_XL) & 3
                assert cl != t
                act = BIT_MASK[cl]
            elif code < OPC_DENSE:
                kind, t = "anti", code & 3
            else:
                kind, t = "dense", code & 3
                m = m + op["lo"].astype(np.complex128)
                if code < OPC_CDENSE:
                    assert fbit == 255 and act == 0xFFFF
            for j in range(16):
                if (j >> t) & 1:
                    a[:, j] *= pend[:, t]
            pend[:, t] = 1.0
            for p in range(8):
                j0 = ((p >> t) << (t + 1)) | (p & ((1 << t) - 1))
                j1 = j0 | (1 << t)
                if not (act >> j0) & 1:
                    continue
                x0, x1 = a[:, j0].copy(), a[:, j1].copy()
                if kind in ("dense", "h"):
                    y0 = m[0] * x0 + m[1] * x1
                    y1 = m[2] * x0 + m[3] * x1
                elif kind == "x":
                    y0, y1 = x1, x0
                else:
                    y0, y1 = m[1] * x1, m[2] * x0
                a[far_on, j0] = y0[far_on]
                a[far_on, j1] = y1[far_on]
        for b in range(4):
            for j in range(16):
                if (j >> b) & 1:
                    a[:, j] *= pend[:, b]
        a *= sc[:, None] * float(ps["scale"])
        st[idx] = a
    if on_pass is not None:
        on_pass(len(passes), None, st)
    # output map: physical index of logical y = map[16] ^ XOR of map[q] over y's set bits
    i = np.arange(1 << n, dtype=np.int64)
    phys = np.full_like(i, int(pos[16]))
    for q in range(n):
        phys ^= ((i >> q) & 1) * int(pos[q])
    return st[phys] * out_scale


def compiled(n, ops):
    c = B.circuit_from_ops(n, ops)
    try:
        return B.tqs_circuit_program(c)
    finally:
        B.tqs_circuit_destroy(c)


CASES = [("bell", 2, W.bell())]
CASES += [(f"ghz{n}", n, W.ghz_chain(n)) for n in (1, 3, 5, 11)]
CASES += [(f"ghzfan{n}", n, W.ghz_fanout(n)) for n in (4, 9)]
CASES += [(f"qft{n}", n, W.qft_on_basis(n, (5 * n + 3) % (1 << n))) for n in (1, 2, 3, 4, 5, 7, 10, 11)]
CASES += [(f"dj{n}{b}", n, W.deutsch_jozsa(n, b, (5, n, int(b)))) for n in (3, 6, 11) for b in (False, True)]
CASES += [(f"rand{n}_{k}", n, W.random_small(n, 8 * n, (6, n, k))) for n in (1, 2, 3, 4, 5, 6, 8) for k in range(3)]
CASES += [(f"mixed{n}", n, W.random_mixed(n, 12, (7, n))) for n in (4, 7, 9, 12)]
CASES += [(f"layered{n}", n, W.random_layered(n, 3, (8, n))) for n in (5, 10, 12)]


def cnot_fan(n, seed):
    """H on every qubit, then CNOTs from a seeded subset of qubits into one target,
    with X gates on the target among them, then H again: runs of exchanges on one
    position with local and far controls (merged into one parity op)."""
    g = W.rng(9, n, seed)
    t = int(g.integers(0, n))
    ops = [("h", (q,), ()) for q in range(n)]
    for c in range(n):
        if c != t and g.random() < 0.6:
            ops.append(("cx", (c, t), ()))
        if g.random() < 0.2:
            ops.append(("x", (t,), ()))
    ops += [("h", (q,), ()) for q in range(n) if q != t]
    return ops


CASES += [(f"fan{n}_{k}", n, cnot_fan(n, k)) for n in (5, 9, 12) for k in range(2)]


@pytest.mark.parametrize("name,n,ops", CASES, ids=[c[0] for c in CASES])
def test_program_replay_matches_oracle(name, n, ops):
    passes, prog_ops, pos, osc, gen = compiled(n, ops)
    got = replay(n, passes, prog_ops, pos, osc, gen)
    want = fsv_route.simulate(n, ops)
    # the program stores matrices in FP32; the replay computes in FP64
    assert np.max(np.abs(got - want)) < 2e-6


def support_tracker(nint, gen):
    """The fused kernel's zero-group rule, checked on the replay: before each
    pass, every amplitude whose physical index differs from the start index
    gen in a bit outside T (the union of the local positions of the register
    passes so far; all bits after a measure / reset or a custom unitary) is
    exactly zero.  Returns the hook and a list of (pass, live amplitudes)."""
    allb = (1 << nint) - 1
    idx = np.arange(1 << nint)
    touched = [0]
    seen = []

    def on_pass(pi, L, st):
        if touched[0] != -1:
            outside = ((idx ^ gen) & allb & ~touched[0]) != 0
            assert np.all(st[outside] == 0), (pi, int(np.count_nonzero(st[outside])))
            seen.append((pi, int(np.count_nonzero(~outside))))
        if L is None:
            return
        if L[0] in (254, 255):
            touched[0] = -1
        elif touched[0] != -1:
            touched[0] |= sum(1 << b for b in L)

    return on_pass, seen


@pytest.mark.parametrize("name,n,ops", CASES, ids=[c[0] for c in CASES])
def test_zero_groups_of_a_basis_start(name, n, ops):
    """What the fused kernel skips is zero: checked pass by pass on the replay
    of the compiled program (the kernel works only the groups that can hold a
    nonzero amplitude, and the generation pass starts from zeros)."""
    passes, prog_ops, pos, osc, gen = compiled(n, ops)
    on_pass, seen = support_tracker(max(n, 4), gen)
    got = replay(n, passes, prog_ops, pos, osc, gen, on_pass=on_pass)
    assert np.max(np.abs(got - fsv_route.simulate(n, ops))) < 2e-6
    assert seen[0] == (0, 1)  # the generation pass works the start state's group only


@pytest.mark.parametrize("n,seed", [(3, 0), (5, 1), (8, 2), (11, 0)])
def test_zero_groups_stop_at_an_instruction(n, seed):
    """After a measure / reset the rule no longer applies (the kernel works
    every group from there on); before it, it holds as above."""
    ops = with_instructions(n, 100 * n + seed)
    u = safe_uniforms(n, ops, seed)
    passes, prog_ops, pos, osc, gen = compiled(n, ops)
    on_pass, seen = support_tracker(max(n, 4), gen)
    replay(n, passes, prog_ops, pos, osc, gen, uniforms=u, outcomes=[], on_pass=on_pass)
    first_instr = next(i for i, p in enumerate(passes) if int(p["L"][0]) == 255)
    assert [pi for pi, _ in seen] == list(range(first_instr + 1))


def test_steps_are_asap():
    """Step table (Sec. 5.2 reading: as soon as possible) matches the oracle's packing."""
    for n, ops in [(2, W.bell()), (6, W.qft(6)), (7, W.random_small(7, 40, (9, 1)))]:
        c = B.circuit_from_ops(n, ops)
        try:
            steps = B.tqs_circuit_steps(c)
            nn, ng, ns = B.tqs_circuit_info(c)
        finally:
            B.tqs_circuit_destroy(c)
        ref = kron_route.steps_asap(n, ops)
        assert ns == len(ref) and ng == len(ops) and nn == n
        k = 0
        want = {}
        for si, st in enumerate(ref):
            for op in st:
                want.setdefault(id(op), si)
        # the oracle keeps op objects; map by position in the input list
        pos_of = {id(op): i for i, op in enumerate(ops)}
        ref_steps = [0] * len(ops)
        for si, st in enumerate(ref):
            for op in st:
                ref_steps[pos_of[id(op)]] = si
        assert steps == ref_steps


def test_ghz_steps_and_passes():
    """GHZ chain on n qubits: n steps.  The CNOT chain is the circuit's
    permutation tail: it is folded into the output map, so the program is the
    one Hadamard on q0 (one pass) and the map sends logical y to the physical
    index whose bit k is y_k ^ y_{k-1} (the inverse of the prefix parities the
    chain computes)."""
    n = 11
    c = B.circuit_from_ops(n, W.ghz_chain(n))
    try:
        assert B.tqs_circuit_info(c)[2] == n
        passes, ops, out_map, osc, gen = B.tqs_circuit_program(c)
        assert len(ops) == 1 and len(passes) == 1 and gen == 0
        # the one unscaled Hadamard's 2^-1/2 sits in the last pass's scale
        assert ops[0]["code"] == OPC_H and osc == 1.0
        assert float(passes[0]["scale"]) == float(np.float32(2 ** -0.5))
        assert int(out_map[16]) == 0
        for q in range(n):
            want = (1 << q) | ((1 << (q + 1)) if q + 1 < n else 0)
            assert int(out_map[q]) == want, q
    finally:
        B.tqs_circuit_destroy(c)


def test_permutation_tail_only_when_last():
    """A CNOT followed by a non-permutation gate on one of its qubits stays in
    the program; X, CNOT and SWAP after every other gate on their qubits are
    folded into the output map."""
    n = 3
    kept = compiled(n, [("h", (0,), ()), ("cx", (0, 1), ()), ("h", (1,), ())])
    folded = compiled(n, [("h", (0,), ()), ("h", (2,), ()), ("cx", (0, 1), ()), ("x", (2,), ()),
                          ("swap", (1, 2), ())])
    assert any(OPC_XF <= int(o["code"]) < OPC_ANTI for o in kept[1])
    assert all(int(o["code"]) < OPC_X or int(o["code"]) == OPC_HMASK for o in folded[1])
    assert int(folded[2][16]) != 0  # the X on q2 is the map's offset


def test_hadamards_grouped_into_one_op():
    """Hadamards of a pass move later past ops on other local positions and
    meet in one OPC_HMASK op; never past an op on their own position.  The
    Deutsch-Jozsa (balanced) program at n = 11 shrinks to 10 ops or fewer; every
    program's replay still matches the oracle (test_program_replay_matches_oracle)."""
    ops = W.deutsch_jozsa(11, True, (1, 3, 2))
    passes, pops, pos, osc, gen = compiled(11, ops)
    codes = [int(o["code"]) for o in pops]
    assert OPC_HMASK in codes
    assert len(pops) <= 10
    # H(0) S(0) H(1): the phase on position 0 is deferred to the end of the pass,
    # so the Hadamards meet, and the phase stays after the Hadamard on its position
    passes, pops, _, _, _ = compiled(2, [("h", (0,), ()), ("s", (0,), ()), ("h", (1,), ())])
    seq = [(int(o["code"]), int(o["t"])) for o in pops]
    assert seq[0] == (OPC_HMASK, 3) and len(seq) == 2 and seq[1][0] >= 40
    # a phase on position 0 between H(0) and a second H(0): nothing is grouped
    # across it (the two stay in order around it)
    passes, pops, _, _, _ = compiled(2, [("h", (0,), ()), ("t", (0,), ()), ("h", (0,), ()),
                                         ("h", (1,), ())])
    assert all(int(o["code"]) != OPC_HMASK or not (int(o["t"]) & 1) for o in pops[:1])
    # the oracle's CNOT fan into the ancilla: one exchange op under a parity
    passes, pops, _, _, _ = compiled(11, ops)
    assert sum(int(o["code"]) == OPC_XP for o in pops) == 1
    assert not any(OPC_XF <= int(o["code"]) < OPC_ANTI for o in pops)
    # two Hadamards on different qubits with nothing between: one op
    passes, pops, _, _, _ = compiled(3, [("h", (0,), ()), ("h", (1,), ()), ("h", (2,), ())])
    assert len(pops) == 1 and int(pops[0]["code"]) == OPC_HMASK and int(pops[0]["t"]) == 7


@pytest.mark.parametrize("bad,status", [
    (("h", (3,), ()), "TQS_ERR_QUBIT_RANGE"),
    (("h", (-1,), ()), "TQS_ERR_QUBIT_RANGE"),
    (("cx", (1, 1), ()), "TQS_ERR_QUBIT_DUP"),
    (("cx", (1,), ()), "TQS_ERR_ARG"),
    (("rx", (0,), ()), "TQS_ERR_ARG"),
    (("cu", (0, 1), (1, 0, 0, 0, 0, 0, 2, 0)), "TQS_ERR_ARG"),
    (("rz", (0,), (float("nan"),)), "TQS_ERR_ARG"),
])
def test_gate_preconditions(bad, status):
    """Preconditions are checked when an operation is added (Sec. 5.2)."""
    c = B.tqs_circuit_create(3)
    try:
        with pytest.raises(B.TqsError) as e:
            B.tqs_add_gate(c, bad[0], bad[1], bad[2])
        assert e.value.name == status
        assert B.tqs_circuit_info(c)[1] == 0
    finally:
        B.tqs_circuit_destroy(c)


def test_circuit_size_limits():
    """Circuits go up to 34 qubits (full-state-vector backend); the fused
    forms and batches stop at 16."""
    with pytest.raises(B.TqsError) as e:
        B.tqs_circuit_create(35)
    assert e.value.name == "TQS_ERR_TOO_MANY_QUBITS"
    c = B.circuit_from_ops(17, W.ghz_chain(17))
    try:
        with pytest.raises(B.TqsError) as e:
            B.tqs_batch_create([c])
        assert e.value.name == "TQS_ERR_TOO_MANY_QUBITS"
        with pytest.raises(B.TqsError) as e:
            B.tqs_circuit_program(c)
        assert e.value.name == "TQS_ERR_TOO_MANY_QUBITS"
    finally:
        B.tqs_circuit_destroy(c)
    with pytest.raises(B.TqsError) as e:
        B.tqs_circuit_create(0)
    assert e.value.name == "TQS_ERR_ARG"


def test_packed_batch_host_side():
    """tqs_batch_create_packed checks preconditions and lays out outputs."""
    circs = [(3, W.ghz_chain(3)), (5, W.qft(5)), (12, W.ghz_chain(12)), (15, W.ghz_chain(15))]
    b = B.tqs_batch_create_packed(*B.pack_ops(circs))
    try:
        count, total, offs = B.tqs_batch_info(b)
        assert count == 4 and total == 8 + 32 + 4096 + 32768
        assert list(offs) == [0, 8, 40, 4136, 36904]
    finally:
        B.tqs_batch_destroy(b)
    nq, off, kind, qub, par = B.pack_ops([(3, [("cx", (0, 3), ())])])
    with pytest.raises(B.TqsError) as e:
        B.tqs_batch_create_packed(nq, off, kind, qub, par)
    assert e.value.name == "TQS_ERR_QUBIT_RANGE"


def test_library_exports_every_declared_symbol():
    """libtqs.so loads on the CPU and exports every function include/tqs.h declares."""
    L = B.lib()
    names = B.header_functions()
    assert len(names) >= 20
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_server_host_side():
    """Server request validation and budget admission, on the host only."""
    sv = B.tqs_server_create(1 << 30, 2, 16)
    try:
        B.tqs_server_submit_packed(sv, 0, 5, B.pack_request(W.ghz_chain(5)))
        B.tqs_server_submit_packed(sv, 1, 16, B.pack_request(W.qft(16)))
        assert B.tqs_server_stats(sv)["queued"] == 2
        with pytest.raises(B.TqsError) as e:
            B.tqs_server_submit_packed(sv, 2, 3, B.pack_request([("cx", (0, 3), ())]))
        assert e.value.name == "TQS_ERR_QUBIT_RANGE"
        with pytest.raises(B.TqsError) as e:
            B.tqs_server_take(sv, 0)
        assert e.value.name == "TQS_ERR_STATE"
    finally:
        B.tqs_server_destroy(sv)
    small = B.tqs_server_create(1 << 16, 1, 4)
    try:
        with pytest.raises(B.TqsError) as e:
            B.tqs_server_submit_packed(small, 0, 14, B.pack_request(W.ghz_chain(14)))
        assert e.value.name == "TQS_ERR_BUDGET"
    finally:
        B.tqs_server_destroy(small)
    with pytest.raises(B.TqsError):
        B.tqs_server_create(0, 1, 1)


def test_launch_options():
    old = B.tqs_get_option(B.OPT_WARPS_PER_CTA, 11)
    try:
        B.tqs_set_option(B.OPT_WARPS_PER_CTA, 11, 8)
        assert B.tqs_get_option(B.OPT_WARPS_PER_CTA, 11) == 8
        for bad in [(11, 0), (11, 17), (3, 4), (12, 4)]:
            with pytest.raises(B.TqsError):
                B.tqs_set_option(B.OPT_WARPS_PER_CTA, *bad)
        with pytest.raises(B.TqsError):
            B.tqs_set_option(99, 11, 4)
        B.tqs_set_option(B.OPT_TEAM_WARPS, 11, 2)
        assert B.tqs_get_option(B.OPT_TEAM_WARPS, 11) == 2
        for bad in [(11, 0), (11, 3), (3, 1), (12, 2)]:
            with pytest.raises(B.TqsError):
                B.tqs_set_option(B.OPT_TEAM_WARPS, *bad)
    finally:
        B.tqs_set_option(B.OPT_WARPS_PER_CTA, 11, old)
        B.tqs_set_option(B.OPT_TEAM_WARPS, 11, 1)


def test_leading_x_gates_fold_into_the_start_state():
    """QFT on a basis state: the preparing X gates cost no op and no pass."""
    n, x = 11, 0b10010110101
    bare = compiled(n, W.qft(n))
    prep = compiled(n, W.qft_on_basis(n, x))
    assert prep[4] == x and bare[4] == 0
    assert len(prep[1]) == len(bare[1]) and len(prep[0]) == len(bare[0])


# ------------------------------------------------ measure / reset instructions

MEAS_CASES = [(n, s) for n in (1, 2, 3, 5, 8, 11) for s in range(3)]


@pytest.mark.parametrize("n,seed", MEAS_CASES)
def test_program_replay_with_instructions_matches_oracle(n, seed):
    ops = with_instructions(n, 100 * n + seed)
    u = safe_uniforms(n, ops, seed)
    passes, prog_ops, pos, osc, gen = compiled(n, ops)
    marks = [int(p["op_begin"]) for p in passes if int(p["L"][0]) == 255]
    assert marks == list(range(len(u)))
    outs = []
    got = replay(n, passes, prog_ops, pos, osc, gen, uniforms=u, outcomes=outs)
    want, want_outs = collapse.simulate_measured(n, ops, u)
    assert [b for _, b in outs] == want_outs
    assert np.max(np.abs(got - want)) < 2e-6


def test_instruction_is_a_barrier_step():
    ops = [("h", (0,), ()), ("h", (1,), ()), ("measure", (0,), ()), ("h", (2,), ()),
           ("x", (1,), ())]
    c = B.circuit_from_ops(3, ops)
    try:
        assert B.tqs_circuit_steps(c) == [0, 0, 1, 2, 2]
        assert B.tqs_circuit_info(c)[2] == 3
    finally:
        B.tqs_circuit_destroy(c)


def test_instruction_reads_the_relabelled_bit():
    """After SWAP(0, 2) the logical qubit 0 lives on physical bit 2."""
    passes, _, pos, _, _ = compiled(3, [("h", (1,), ()), ("swap", (0, 2), ()), ("measure", (0,), ())])
    ins = [p for p in passes if int(p["L"][0]) == 255]
    assert len(ins) == 1 and int(ins[0]["L"][1]) == 2 and int(pos[0]) == 1 << 2


def test_unitary_forms_reject_instructions():
    ops = [("h", (0,), ()), ("measure", (0,), ())]
    c = B.circuit_from_ops(2, ops)
    try:
        for call in (lambda: B.tqs_simulate(c, None, stream=0),
                     lambda: B.tqs_simulate_plain(c, None, stream=0),
                     lambda: B.tqs_circuit_unitary(c, B.PREC_FP32_SIMT, None, stream=0)):
            with pytest.raises(B.TqsError) as e:
                call()
            assert e.value.name == "TQS_ERR_UNSUPPORTED"
    finally:
        B.tqs_circuit_destroy(c)
    b = B.tqs_batch_create_packed(*B.pack_ops([(2, ops), (3, W.ghz_chain(3)), (2, ops + ops)]))
    try:
        assert B.tqs_batch_instructions(b).tolist() == [0, 1, 1, 3]
        with pytest.raises(B.TqsError) as e:
            B.tqs_batch_run(b, None, stream=0)
        assert e.value.name == "TQS_ERR_UNSUPPORTED"
    finally:
        B.tqs_batch_destroy(b)
    sv = B.tqs_server_create(1 << 30, 1, 4)
    try:
        with pytest.raises(B.TqsError) as e:
            B.tqs_server_submit_packed(sv, 0, 2, B.pack_request(ops))
        assert e.value.name == "TQS_ERR_UNSUPPORTED"
    finally:
        B.tqs_server_destroy(sv)


# ------------------------------------------------------------ custom unitaries

def rand_unitary(k, seed):
    rng = np.random.default_rng(seed)
    a = rng.normal(size=(1 << k, 1 << k)) + 1j * rng.normal(size=(1 << k, 1 << k))
    q, r = np.linalg.qr(a)
    return q * (np.diag(r) / np.abs(np.diag(r)))


def with_customs(n, seed):
    """Random circuit with custom unitaries of k = 1..min(5, n) spliced in,
    one of them after a SWAP (so its qubits are relabelled)."""
    from oracle import gates as G
    rng = np.random.default_rng(seed)
    ops = list(W.random_small(n, 4 * n, (12, n, seed)))
    mats = []
    for j, k in enumerate(range(1, min(5, n) + 1)):
        qs = tuple(int(q) for q in rng.permutation(n)[:k])
        m = rand_unitary(k, 10 * seed + k)
        at = int(rng.integers(0, len(ops) + 1))
        ins = [("unitary", qs, G.custom_params(m))]
        if j == 1 and n >= 2:
            ins = [("swap", (qs[0], (qs[0] + 1) % n), ())] + ins
        ops[at:at] = ins
        if k >= 2:
            mats.append((at, m))
    # wide customs appear in the program in circuit order
    order = [op for op in ops if op[0] == "unitary" and len(op[1]) >= 2]
    return ops, [G.custom_matrix(op[1], op[2]) for op in order]


@pytest.mark.parametrize("n,seed", [(n, s) for n in (2, 3, 5, 7, 11) for s in range(2)])
def test_program_replay_with_customs_matches_oracle(n, seed):
    ops, mats = with_customs(n, 40 * n + seed)
    passes, prog_ops, pos, osc, gen = compiled(n, ops)
    assert sum(1 for p in passes if int(p["L"][0]) == 254) == len(mats)
    got = replay(n, passes, prog_ops, pos, osc, gen, customs=mats)
    want = fsv_route.simulate(n, ops)
    assert np.max(np.abs(got - want)) < 2e-6


def test_custom_registry_errors():
    m = rand_unitary(2, 1)
    B.tqs_register_unitary("reg_test_u2", m)
    c = B.tqs_circuit_create(4)
    try:
        B.tqs_add_custom(c, "reg_test_u2", (3, 1))
        for args, status in [(("no_such_name", (0, 1)), "TQS_ERR_ARG"),
                             (("reg_test_u2", (0, 1, 2)), "TQS_ERR_ARG"),
                             (("reg_test_u2", (0, 4)), "TQS_ERR_QUBIT_RANGE"),
                             (("reg_test_u2", (2, 2)), "TQS_ERR_QUBIT_DUP")]:
            with pytest.raises(B.TqsError) as e:
                B.tqs_add_custom(c, *args)
            assert e.value.name == status
        assert B.tqs_circuit_info(c)[1] == 1
    finally:
        B.tqs_circuit_destroy(c)
    bad = m.copy()
    bad[0, 0] += 1e-6
    with pytest.raises(B.TqsError) as e:
        B.tqs_register_unitary("reg_test_bad", bad)
    assert e.value.name == "TQS_ERR_ARG"
    with pytest.raises(B.TqsError):
        B.tqs_register_unitary("reg_test_big", np.eye(64))


# ------------------------------------------------------- full state vector

def test_fsv_pass_grouping():
    """GHZ chain, CNOT targets 1..n-1.  At n = 20 tiles hold the 5 lowest bits
    plus 7 more (2^12 amplitudes below 24 qubits), so targets 1..11 share the
    first pass, 12..18 the second and 19 the third; at n = 30 (2^13-amplitude
    tiles: 8 more bits) 1..12, 13..20 and 21..28 take a pass each, 29 the last."""
    c = B.circuit_from_ops(30, W.ghz_chain(30))
    try:
        assert B.tqs_fsv_passes(c) == (4, 13)
    finally:
        B.tqs_circuit_destroy(c)
    c = B.circuit_from_ops(20, W.ghz_chain(20))
    try:
        assert B.tqs_fsv_passes(c) == (3, 12)
    finally:
        B.tqs_circuit_destroy(c)
    # diagonal gates and controls never need a tile slot
    ops = [("h", (0,), ())] + [("cp", (19, q), (0.3,)) for q in range(5)] + [("z", (18,), ())]
    c = B.circuit_from_ops(20, ops)
    try:
        assert B.tqs_fsv_passes(c) == (1, 12)
    finally:
        B.tqs_circuit_destroy(c)


def test_fsv_gates_per_pass_option():
    """TQS_OPT_FSV_MAX_GATES = 1 is the per-gate form (one pass per gate);
    the cached passes follow the option; bad keys and values are refused."""
    ops = W.random_layered(16, 2, (19, 16))
    c = B.circuit_from_ops(16, ops)
    try:
        grouped = B.tqs_fsv_passes(c)[0]
        B.tqs_set_option(B.OPT_FSV_MAX_GATES, 0, 1)
        assert B.tqs_get_option(B.OPT_FSV_MAX_GATES, 0) == 1
        assert B.tqs_fsv_passes(c)[0] == len(ops)
        B.tqs_set_option(B.OPT_FSV_MAX_GATES, 0, 5)
        assert B.tqs_fsv_passes(c)[0] >= -(-len(ops) // 5)
    finally:
        B.tqs_set_option(B.OPT_FSV_MAX_GATES, 0, 0)
        B.tqs_circuit_destroy(c)
    assert grouped < len(ops)
    for key, value in ((1, 1), (0, -1)):
        with pytest.raises(B.TqsError) as e:
            B.tqs_set_option(B.OPT_FSV_MAX_GATES, key, value)
        assert e.value.name == "TQS_ERR_ARG"


def test_exact_probs_option():
    assert B.tqs_get_option(B.OPT_EXACT_PROBS, 0) == 0
    try:
        B.tqs_set_option(B.OPT_EXACT_PROBS, 0, 1)
        assert B.tqs_get_option(B.OPT_EXACT_PROBS, 0) == 1
        for key, value in ((1, 1), (0, 2)):
            with pytest.raises(B.TqsError) as e:
                B.tqs_set_option(B.OPT_EXACT_PROBS, key, value)
            assert e.value.name == "TQS_ERR_ARG"
    finally:
        B.tqs_set_option(B.OPT_EXACT_PROBS, 0, 0)


def test_host_writes_option():
    assert B.tqs_get_option(B.OPT_HOST_WRITES, 0) == 1
    try:
        B.tqs_set_option(B.OPT_HOST_WRITES, 0, 0)
        assert B.tqs_get_option(B.OPT_HOST_WRITES, 0) == 0
        for key, value in ((1, 1), (0, 2)):
            with pytest.raises(B.TqsError) as e:
                B.tqs_set_option(B.OPT_HOST_WRITES, key, value)
            assert e.value.name == "TQS_ERR_ARG"
    finally:
        B.tqs_set_option(B.OPT_HOST_WRITES, 0, 1)


def test_multi_cta_option():
    assert B.tqs_get_option(B.OPT_MULTI_CTAS, 0) == 8
    try:
        for v in (0, 1, 3, 64):
            B.tqs_set_option(B.OPT_MULTI_CTAS, 0, v)
            assert B.tqs_get_option(B.OPT_MULTI_CTAS, 0) == v
        for key, value in ((1, 2), (0, -1), (0, 65)):
            with pytest.raises(B.TqsError) as e:
                B.tqs_set_option(B.OPT_MULTI_CTAS, key, value)
            assert e.value.name == "TQS_ERR_ARG"
    finally:
        B.tqs_set_option(B.OPT_MULTI_CTAS, 0, 8)


def test_large_circuits_only_in_fsv():
    c = B.tqs_circuit_create(34)
    try:
        B.tqs_add_gate(c, "h", (33,))
        with pytest.raises(B.TqsError) as e:
            B.tqs_simulate(c, None, stream=0)
        assert e.value.name == "TQS_ERR_TOO_MANY_QUBITS"
        assert B.tqs_fsv_passes(c)[0] == 1
    finally:
        B.tqs_circuit_destroy(c)
    with pytest.raises(B.TqsError):
        B.tqs_circuit_create(35)


@pytest.mark.filterwarnings("ignore::DeprecationWarning")
def test_host_pool_survives_fork():
    """Batch creation runs on a persistent pool of host threads; a child
    process forked after the pool exists gets a pool of its own (the parent's
    threads do not exist there) and creates batches normally."""
    import os
    circs = [(n, W.random_mixed(n, 6, (17, n, i))) for i, n in enumerate([5, 9, 11, 12] * 64)]
    arrays = B.pack_ops(circs)
    b = B.tqs_batch_create_packed(*arrays)   # starts the pool in this process
    count0 = B.tqs_batch_info(b)[0]
    B.tqs_batch_destroy(b)
    pid = os.fork()
    if pid == 0:
        code = 1
        try:
            bb = B.tqs_batch_create_packed(*arrays)
            code = 0 if B.tqs_batch_info(bb)[0] == count0 else 2
            B.tqs_batch_destroy(bb)
        finally:
            os._exit(code)
    _, status = os.waitpid(pid, 0)
    assert os.WIFEXITED(status) and os.WEXITSTATUS(status) == 0
    b = B.tqs_batch_create_packed(*arrays)
    assert B.tqs_batch_info(b)[0] == count0
    B.tqs_batch_destroy(b)


# ------------------------------------------------ allocator and cancellation

def test_allocator_failure_is_nomem():
    """A caller allocator that refuses memory fails the call with
    TQS_ERR_NOMEM before any device work (host-side fault injection)."""
    calls = []

    def refuse(n, stream):
        calls.append(n)
        return 0

    B.tqs_set_allocator(refuse, lambda p, s: None)
    try:
        c = B.circuit_from_ops(5, W.ghz_chain(5))
        try:
            st = B.lib().tqs_simulate(c, None, 256, None, None, None)
            assert B.STATUS[st] == "TQS_ERR_NOMEM" and calls
            st = B.lib().tqs_circuit_unitary(c, B.PREC_FP32_SIMT, 256, None)
            assert B.STATUS[st] == "TQS_ERR_NOMEM"
        finally:
            B.tqs_circuit_destroy(c)
        b = B.tqs_batch_create_packed(*B.pack_ops([(6, W.ghz_chain(6))] * 4))
        try:
            st = B.lib().tqs_batch_run(b, 256, None, None, 0, None)
            assert B.STATUS[st] == "TQS_ERR_NOMEM"
        finally:
            B.tqs_batch_destroy(b)
        st = B.lib().tqs_probabilities(256, 10, None, 512, None)
        assert B.STATUS[st] == "TQS_ERR_NOMEM"
    finally:
        B.tqs_set_allocator()
    # one callback without the other is an argument error
    assert B.STATUS[B.lib().tqs_set_allocator(B.ALLOC_FN(lambda n, s, c: None), None, None)] == "TQS_ERR_ARG"


def test_server_cancel_host_side():
    sv = B.tqs_server_create(1 << 30, 1, 8)
    try:
        for tag in range(3):
            B.tqs_server_submit_packed(sv, tag, 5, B.pack_request(W.ghz_chain(5)))
        B.tqs_server_cancel(sv, 1)
        assert B.tqs_server_stats(sv)["queued"] == 2
        for tag, status in ((1, "TQS_ERR_ARG"), (7, "TQS_ERR_ARG")):
            with pytest.raises(B.TqsError) as e:
                B.tqs_server_cancel(sv, tag)
            assert e.value.name == status
    finally:
        B.tqs_server_destroy(sv)


def test_launch_shape_options_validated():
    """The autotuner's options take their documented ranges only (host check)."""
    for opt, good, bad in [(B.OPT_CTA_THREADS, (256, 512), (128, 300, 1024)),
                           (B.OPT_FSV_TILE_Q, (0, 10, 13), (9, 14, -1)),
                           (B.OPT_CHAIN_GROUP, (1, 16, 64), (0, 65)),
                           (B.OPT_CHAIN_KCHUNK, (0, 64, 512, 1 << 20), (-64, 32, 100, (1 << 20) + 64)),
                           (B.OPT_CHAIN_PAIR, (0, 1), (-1, 2))]:
        old = B.tqs_get_option(opt, 0)
        try:
            for v in good:
                B.tqs_set_option(opt, 0, v)
                assert B.tqs_get_option(opt, 0) == v
            for v in bad:
                with pytest.raises(B.TqsError):
                    B.tqs_set_option(opt, 0, v)
            with pytest.raises(B.TqsError):
                B.tqs_set_option(opt, 1, good[0])
        finally:
            B.tqs_set_option(opt, 0, old)


def test_asap_steps_matches_library_step_count():
    """workloads.asap_steps (the bench reference arm's step count, pure Python)
    equals the library's ASAP step table (tqs_batch_info's total steps)."""
    mix = W.paper_mix(11, 48, seed_tag=5) + [("r", W.random_mixed(7, 9, (5, 1)))]
    circs = [(11, ops) for _, ops in mix[:-1]] + [(7, mix[-1][1])]
    b = B.tqs_batch_create_packed(*B.pack_ops(circs))
    try:
        steps = B.tqs_batch_info(b, extra=True)[3]
    finally:
        B.tqs_batch_destroy(b)
    assert steps == sum(W.asap_steps(ops) for _, ops in circs)


def test_cta_threads_tuning_keys_tell_batches_apart():
    """The one-CTA team's thread count is tuned per subset of 12..14-qubit
    circuits: the mixed random batch and the all-14-qubit batch (same size,
    same largest n) must not share a cached choice."""
    from paper_2305_14398_gb300 import autotune
    mixed = W.batch_circuits(4096, seed_tag=3)
    n14 = W.batch_circuits_fixed_n(4096, 14, seed_tag=5)
    sub_m, key_m = autotune.cta_subset(mixed)
    sub_14, key_14 = autotune.cta_subset(n14)
    assert len(sub_14) == 4096
    assert 0 < len(sub_m) < 4096
    assert all(12 <= n <= 14 for n, _ in sub_m)
    assert key_m != key_14
    assert autotune.cta_subset([(8, [("h", [0], [])])]) == ([], "cta|0|a0|g0")


def test_bench_reports_traffic_only_for_the_captured_shape():
    """roofline.traffic is the ncu capture's DRAM bytes, and only when the bench
    times the launch shape that capture was taken at."""
    import bench
    cap = {"team_warps": 1, "warps_per_cta": 1, "bytes": 123}
    assert bench.roofline_traffic(1, 1, cap) == 123
    assert bench.roofline_traffic(2, 8, cap) is None
    assert bench.roofline_traffic(1, 8, cap) is None
    assert bench.roofline_traffic(1, 1, None) is None
    c = bench.NCU_TRAFFIC
    if c is not None:  # the committed capture: DRAM bytes of one launch, within the outputs
        assert 0 < c["bytes"] <= 16384 * (16 << 11) + (64 << 20)
