"""CKKS circuits as DAGs of library operations, for request serving.

A circuit is built once per query shape: every node is one library
operation (subtract, add, HMult+relin+rescale, multiply by an integer,
add a constant, rescale, drop levels, rotate) with its level and its CKKS
scale worked out at build time.  Nodes are grouped into stages by
dependency depth; a request runs one stage at a time, and the serving loop
(serving.py) submits the current stage of every active request as one
uneven batch, so requests overlap on the GPU.

Scales: inputs carry the scale `delta`; a real constant c multiplies as the
integer round(c q) followed by a rescale by that same prime q, which keeps
the scale; a ciphertext product ends at scale s_a s_b / q.  The float64
evaluator (`evaluate_float`) runs the same circuit on plaintext arrays with
the same integer constants, so the decrypted result can be compared with it.

The polynomial evaluator follows the baby-step / giant-step scheme in the
Chebyshev basis: p = q T_n + r with n the largest power of two not above
deg p (using T_n T_m = (T_{n+m} + T_{|n-m|}) / 2), recursively, down to
leaves of degree < 8 evaluated from T_1 .. T_7 by integer products, one
rescale and one constant.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

from . import api


@dataclass
class Node:
    id: int
    kind: str                 # input sub add mul mul_int rescale add_const drop rotate
    args: tuple = ()
    level: int = 0
    scale: float = 1.0
    const: int = 0            # mul_int / add_const integer constant
    kscale: float = 1.0       # mul_int: the scale the integer constant stands at
    galois: int = 0           # rotate: Galois element
    steps: int = 0            # rotate: slot rotation
    name: str = ""
    stage: int = 0


class Circuit:
    def __init__(self, primes, delta: float, log_n: int):
        self.q = list(primes)           # q_0 .. q_{L-1}
        self.delta = delta
        self.log_n = log_n
        self.n = 1 << log_n
        self.nodes: list[Node] = []
        self.inputs: dict[str, int] = {}
        self.outputs: dict[str, int] = {}

    # ------------------------------------------------------------ building
    def _add(self, **kw) -> int:
        node = Node(id=len(self.nodes), **kw)
        if node.args:
            node.stage = 1 + max(self.nodes[a].stage for a in node.args)
        self.nodes.append(node)
        return node.id

    def input(self, name: str, level: int) -> int:
        i = self._add(kind="input", level=level, scale=self.delta, name=name)
        self.inputs[name] = i
        return i

    def output(self, name: str, x: int) -> None:
        self.outputs[name] = x

    def level(self, x: int) -> int:
        return self.nodes[x].level

    def drop(self, x: int, level: int) -> int:
        nd = self.nodes[x]
        if level >= nd.level:
            return x
        return self._add(kind="drop", args=(x,), level=level, scale=nd.scale)

    def _align(self, a: int, b: int):
        lv = min(self.level(a), self.level(b))
        return self.drop(a, lv), self.drop(b, lv)

    def add(self, a: int, b: int) -> int:
        a, b = self._align(a, b)
        return self._add(kind="add", args=(a, b), level=self.level(a), scale=self.nodes[a].scale)

    def sub(self, a: int, b: int) -> int:
        a, b = self._align(a, b)
        return self._add(kind="sub", args=(a, b), level=self.level(a), scale=self.nodes[a].scale)

    def mul(self, a: int, b: int) -> int:
        """HMult + relinearise + rescale."""
        a, b = self._align(a, b)
        lv = self.level(a)
        scale = self.nodes[a].scale * self.nodes[b].scale / self.q[lv - 1]
        return self._add(kind="mul", args=(a, b), level=lv - 1, scale=scale)

    def mul_int(self, a: int, k: int, kscale: float = 1.0) -> int:
        """Times the integer k, read as the real k / kscale (the output scale
        is the input scale times kscale)."""
        nd = self.nodes[a]
        return self._add(kind="mul_int", args=(a,), level=nd.level, scale=nd.scale * kscale,
                         const=int(k), kscale=kscale)

    def rescale(self, a: int) -> int:
        nd = self.nodes[a]
        return self._add(kind="rescale", args=(a,), level=nd.level - 1,
                         scale=nd.scale / self.q[nd.level - 1])

    def scalar(self, a: int, c: float) -> int:
        """Times the real c at unchanged scale: integer round(c q_top), rescale."""
        qt = self.q[self.level(a) - 1]
        return self.rescale(self.mul_int(a, int(round(c * qt)), kscale=qt))

    def add_const(self, a: int, c: float) -> int:
        nd = self.nodes[a]
        k = int(np.sign(c * nd.scale) * np.floor(abs(c * nd.scale) + 0.5))
        return self._add(kind="add_const", args=(a,), level=nd.level, scale=nd.scale, const=k)

    def rotate(self, a: int, steps: int, galois: int) -> int:
        nd = self.nodes[a]
        return self._add(kind="rotate", args=(a,), level=nd.level, scale=nd.scale,
                         galois=galois, steps=steps)

    # ------------------------------------------------------------ polynomials
    def chebyshev(self, x: int, coeffs) -> int:
        """sum_k coeffs[k] T_k(x) for x with values in [-1, 1]."""
        c = [float(v) for v in coeffs]
        while len(c) > 1 and c[-1] == 0.0:
            c.pop()
        deg = len(c) - 1
        T = {1: x}

        def two_t_sq_minus_1(a):          # T_{2a} = 2 T_a^2 - 1
            return self.add_const(self.mul_int(self.mul(T[a], T[a]), 2), -1.0)

        def two_tt_minus_t(a, b, d):      # T_{a+b} = 2 T_a T_b - T_{b-a}
            return self.sub(self.mul_int(self.mul(T[a], T[b]), 2), T[d])

        if deg >= 2:
            T[2] = two_t_sq_minus_1(1)
        if deg >= 3:
            T[3] = two_tt_minus_t(1, 2, 1)
        if deg >= 4:
            T[4] = two_t_sq_minus_1(2)
        if deg >= 5:
            T[5] = two_tt_minus_t(2, 3, 1)
        if deg >= 6:
            T[6] = two_t_sq_minus_1(3)
        if deg >= 7:
            T[7] = two_tt_minus_t(3, 4, 1)
        n = 8
        while n <= deg:
            T[n] = two_t_sq_minus_1(n // 2)
            n *= 2

        def leaf(cs):
            terms = [(k, v) for k, v in enumerate(cs) if k >= 1 and v != 0.0]
            if not terms:
                terms = [(1, 0.0)]
            lv = min(self.level(T[k]) for k, _ in terms)
            qt = self.q[lv - 1]
            acc = None
            for k, v in terms:
                p = self.mul_int(self.drop(T[k], lv), int(round(v * qt)), kscale=qt)
                acc = p if acc is None else self.add(acc, p)
            out = self.rescale(acc)
            if cs[0] != 0.0:
                out = self.add_const(out, cs[0])
            return out

        def rec(cs):
            d = len(cs) - 1
            if d < 8:
                return leaf(cs)
            n = 1
            while n * 2 <= d:
                n *= 2
            qc = [cs[n]] + [2.0 * cs[k] for k in range(n + 1, d + 1)]
            rc = list(cs[:n])
            for k in range(n + 1, d + 1):
                rc[2 * n - k] -= cs[k]
            return self.add(self.mul(rec(qc), T[n]), rec(rc))

        return rec(c)

    # ------------------------------------------------------------ analysis
    def live(self) -> set:
        """Nodes the outputs depend on (the others are never run)."""
        seen, todo = set(), list(self.outputs.values())
        while todo:
            i = todo.pop()
            if i not in seen:
                seen.add(i)
                todo.extend(self.nodes[i].args)
        return seen

    def stages(self) -> list[list[int]]:
        out: dict[int, list[int]] = {}
        live = self.live()
        for nd in self.nodes:
            if nd.kind != "input" and nd.id in live:
                out.setdefault(nd.stage, []).append(nd.id)
        return [out[k] for k in sorted(out)]

    def peak_bytes(self) -> int:
        """Largest total size of live intermediate ciphertexts over the stages."""
        last_use = {}
        alive = self.live()
        for nd in self.nodes:
            if nd.id in alive:
                for a in nd.args:
                    last_use[a] = max(last_use.get(a, 0), nd.stage)
        for o in self.outputs.values():
            last_use[o] = 1 << 30
        live, peak = {}, 0
        for st in self.stages():
            for i in st:
                live[i] = 2 * self.nodes[i].level * self.n * 8
            peak = max(peak, sum(live.values()))
            s = self.nodes[st[0]].stage
            for i in list(live):
                if last_use.get(i, 0) <= s:
                    del live[i]
        return peak

    def counts(self) -> dict:
        """Operations run per request, by kind (live nodes only)."""
        c: dict[str, int] = {}
        live = self.live()
        for nd in self.nodes:
            if nd.id in live:
                c[nd.kind] = c.get(nd.kind, 0) + 1
        return c

    # ------------------------------------------------------------ float reference
    def evaluate_float(self, values: dict[str, np.ndarray]) -> dict[str, np.ndarray]:
        """The same circuit on plaintext slot vectors with the same integer
        constants and scales: node value = message / node scale, so an
        integer k read at scale s multiplies by k / s, a rescale keeps the
        value, a sum weighs the second term by the ratio of the scales."""
        v: dict[int, np.ndarray] = {}
        for nd in self.nodes:
            if nd.kind == "input":
                v[nd.id] = np.asarray(values[nd.name], dtype=np.complex128)
                continue
            a = v[nd.args[0]]
            if nd.kind in ("sub", "add"):
                b = v[nd.args[1]] * (self.nodes[nd.args[1]].scale / self.nodes[nd.args[0]].scale)
                r = a - b if nd.kind == "sub" else a + b
            elif nd.kind == "mul":
                r = a * v[nd.args[1]]
            elif nd.kind == "mul_int":
                r = a * (nd.const / nd.kscale)
            elif nd.kind in ("rescale", "drop"):
                r = a
            elif nd.kind == "add_const":
                r = a + nd.const / nd.scale
            elif nd.kind == "rotate":
                r = np.roll(a, -nd.steps)
            else:
                raise ValueError(nd.kind)
            v[nd.id] = r
        return {k: v[i] for k, i in self.outputs.items()}


_OP_KIND = {"sub": api.OP_SUB, "add": api.OP_ADD, "mul": api.OP_MUL_RELIN_RESCALE,
            "mul_int": api.OP_MUL_INT, "rescale": api.OP_RESCALE, "add_const": api.OP_ADD_CONST,
            "drop": api.OP_DROP, "rotate": api.OP_ROTATE}


@dataclass
class Schedule:
    """Per-stage entries (node id, op kind, argument ids, level, integer
    argument) and the node ids whose buffers may be released after each stage."""
    stages: list
    release: list


def schedule(circuit: Circuit) -> Schedule:
    cached = getattr(circuit, "_schedule", None)
    if cached is not None and cached[0] == len(circuit.nodes):
        return cached[1]
    groups = circuit.stages()
    live = circuit.live()
    last_use: dict[int, int] = {}
    for nd in circuit.nodes:
        if nd.id in live:
            for a in nd.args:
                last_use[a] = max(last_use.get(a, 0), nd.stage)
    keep = set(circuit.outputs.values()) | set(circuit.inputs.values())
    by_stage: dict[int, list] = {}
    for i, s in last_use.items():
        if i not in keep:
            by_stage.setdefault(s, []).append(i)
    stages, release = [], []
    for g in groups:
        entries = []
        for i in g:
            nd = circuit.nodes[i]
            arg = nd.galois if nd.kind == "rotate" else nd.const
            entries.append((i, _OP_KIND[nd.kind], nd.args, nd.level, arg))
        stages.append(entries)
        release.append(by_stage.get(circuit.nodes[g[0]].stage, []))
    sch = Schedule(stages, release)
    circuit._schedule = (len(circuit.nodes), sch)
    return sch


@dataclass
class MemoryPlan:
    """Byte offsets of a circuit's intermediate ciphertexts in one arena per
    request.  A node's buffer is live from its stage to the last stage that
    reads it (outputs: to the end); two nodes share bytes only if one's last
    reader runs in an earlier stage than the other's own stage, so that no
    batch (one stage of many requests) reads memory that it also writes."""
    offsets: dict
    sizes: dict
    live: dict          # node id -> (first stage, last stage)
    size: int


def memory_plan(circuit: Circuit, align: int = 256) -> MemoryPlan:
    """First fit, stage by stage, against the buffers live in that stage."""
    cached = getattr(circuit, "_memory_plan", None)
    if cached is not None and cached[0] == len(circuit.nodes):
        return cached[1]
    alive = circuit.live()
    last = {}
    for nd in circuit.nodes:
        if nd.id in alive:
            for a in nd.args:
                last[a] = max(last.get(a, 0), nd.stage)
    end = 1 << 30
    for o in circuit.outputs.values():
        last[o] = end
    offsets, sizes, live = {}, {}, {}
    for st in circuit.stages():
        s = circuit.nodes[st[0]].stage
        busy = sorted((offsets[i], offsets[i] + sizes[i]) for i in offsets if live[i][1] >= s)
        for i in st:
            size = 2 * circuit.nodes[i].level * circuit.n * 8
            off = 0
            for a, b in busy:
                if a >= off + size:
                    break
                if b > off:
                    off = (b + align - 1) // align * align
            offsets[i], sizes[i], live[i] = off, size, (s, last.get(i, s))
            busy = sorted(busy + [(off, off + size)])
    total = max((offsets[i] + sizes[i] for i in offsets), default=0)
    plan = MemoryPlan(offsets, sizes, live, total)
    circuit._memory_plan = (len(circuit.nodes), plan)
    return plan


class Runner:
    """One request's instance of a circuit: device buffers per node, the
    batch entries of the current stage, and buffer release after last use.

    With `arena` (a device byte tensor of memory_plan(circuit).size bytes)
    every intermediate lives at its planned offset there, and the entries of
    every stage are built once, here: a tick then only gathers them, with no
    allocation or entry marshalling per operation."""

    def __init__(self, circuit: Circuit, ctx, keys, inputs: dict, arena=None):
        self.c = circuit
        self.ctx, self.keys = ctx, keys
        self.buf: dict[int, object] = {}
        for name, i in circuit.inputs.items():
            self.buf[i] = inputs[name]
        self.sch = schedule(circuit)
        self.pos = 0
        self.arena = arena
        self.ops = None
        if arena is not None:
            plan = memory_plan(circuit)
            base = arena.data_ptr()
            ptr = {i: base + off for i, off in plan.offsets.items()}
            for i, t in self.buf.items():
                ptr[i] = t.data_ptr()
            nodes = circuit.nodes
            self.ops = []
            for entries in self.sch.stages:
                ops = []
                for i, kind, args, level, arg in entries:
                    ops.append(api.make_op_ptr(
                        kind, ctx, 1, nodes[args[0]].level, level, ptr[args[0]],
                        ptr[args[1]] if len(args) > 1 else None, ptr[i], keys=keys,
                        galois_elt=arg if kind == api.OP_ROTATE else 0,
                        const=0 if kind == api.OP_ROTATE else arg))
                self.ops.append(ops)

    @property
    def done(self) -> bool:
        return self.pos >= len(self.sch.stages)

    @property
    def remaining(self) -> int:
        return len(self.sch.stages) - self.pos

    def stage_ops(self) -> list:
        if self.ops is not None:
            return self.ops[self.pos]
        ops = []
        for i, kind, args, level, arg in self.sch.stages[self.pos]:
            a = self.buf[args[0]]
            out = self.ctx.empty_ct(a.shape[0], level)
            self.buf[i] = out
            b = self.buf[args[1]] if len(args) > 1 else None
            ops.append(api.make_op(kind, self.ctx, a, out, keys=self.keys, b=b,
                                   galois_elt=arg if kind == api.OP_ROTATE else 0,
                                   const=0 if kind == api.OP_ROTATE else arg))
        return ops

    def advance(self) -> None:
        """Drops the buffers last read by the current stage; call it only
        after that stage has been enqueued."""
        if self.ops is None:
            for i in self.sch.release[self.pos]:
                self.buf.pop(i, None)
        self.pos += 1

    def result(self, name: str):
        i = self.c.outputs[name]
        if self.ops is None:
            return self.buf[i]
        plan = memory_plan(self.c)
        import torch
        words = self.arena.narrow(0, plan.offsets[i], plan.sizes[i]).view(torch.int64)
        return words.view(1, 2, self.c.nodes[i].level, self.c.n)

    def release(self) -> None:
        self.buf.clear()
        self.arena = None
        self.ops = None


def pdq_circuit(ctx, delta: float, coeffs, kappa: float = 1.0, sum_slots: int = 1024,
                galois=None, with_count: bool = False) -> Circuit:
    """The range-predicate masked sum: with x = column a, y = column b and
    encrypted bounds lo, hi,
        u = kappa (x - lo), v = kappa (hi - x),
        mask = (1 + p(u)) (1 + p(v)) / 4,  p ~ sign (Chebyshev coefficients),
        out = sum over slots 0 .. sum_slots-1 of mask * y (rotate-and-add).
    with_count adds the input "ones" (1 in the table's rows) and the output
    "count" = the same sum of mask * ones, for the search-and-average query."""
    c = Circuit(ctx.q, delta, int(np.log2(ctx.n)))
    L = ctx.L
    x, y = c.input("x", L), c.input("y", L)
    lo, hi = c.input("lo", L), c.input("hi", L)
    d1, d2 = c.sub(x, lo), c.sub(hi, x)
    if kappa != 1.0:
        d1, d2 = c.scalar(d1, kappa), c.scalar(d2, kappa)
    pu, pv = c.chebyshev(d1, coeffs), c.chebyshev(d2, coeffs)
    mask = c.mul(c.add_const(pu, 1.0), c.add_const(pv, 1.0))
    mask = c.scalar(mask, 0.25)
    def slot_sum(t):
        r = 1
        while r < sum_slots:
            g = galois[r] if galois is not None else ctx.galois_elt(r)
            t = c.add(t, c.rotate(t, r, g))
            r *= 2
        return t

    c.output("sum", slot_sum(c.mul(mask, y)))
    if with_count:
        ones = c.input("ones", L)
        c.output("count", slot_sum(c.mul(mask, ones)))
    return c
