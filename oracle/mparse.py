"""The oracle's model parser for transition strings (Sec. 3.5, "Using the
model parser to define a new model").

TEST INFRASTRUCTURE ONLY.  Written independently of the CUDA library's
parser: this one turns the strings into the state-change matrix S, the
dependency graph G and C code for the propensities, which gcc compiles into a
shared library that the oracle calls through a function pointer -- the same
route the paper describes (generated C code, compiled, loaded, run).

Transitions are "LHS -> propensity -> RHS" (Sec. 3.5): LHS / RHS are "@" (the
empty set) or compartment names joined by "+" (a name may be preceded by
"k*" to count k times); the propensity is an expression over compartment
names (the node's counts, as double), global data names (gdata), decimal
numbers, "+", "-", "*", "/", unary minus and parentheses, with the usual
precedence and left-to-right grouping.

Readings (the paper shows examples only): S[p, j] = (count of p on the RHS)
- (count on the LHS); G[k, j] = 1 when propensity k reads a compartment that
transition j changes; a name may not be both a compartment and a gdata name;
numbers become the nearest double; each operation is one IEEE double
operation in the written grouping (no contraction), so a propensity means
the same on every conforming machine.  Math functions are not part of the
grammar.
"""
import hashlib
import os
import re
import subprocess
from dataclasses import dataclass

import ctypes
import numpy as np

_DIR = os.path.dirname(os.path.abspath(__file__))
_BUILD = os.path.join(_DIR, "_build")

_TOKEN = re.compile(r"\s*(?:(?P<num>(?:\d+\.?\d*|\.\d+)(?:[eE][+-]?\d+)?)"
                    r"|(?P<name>[A-Za-z_.][A-Za-z0-9_.]*)|(?P<op>[-+*/()]))")


class ParseError(ValueError):
    pass


def _tokens(text):
    pos, out = 0, []
    text = text.rstrip()
    while pos < len(text):
        m = _TOKEN.match(text, pos)
        if not m or m.end() == pos:
            raise ParseError(f"cannot read {text[pos:]!r}")
        pos = m.end()
        for kind in ("num", "name", "op"):
            if m.group(kind) is not None:
                out.append((kind, m.group(kind)))
    return out


class _Expr:
    """Recursive descent over the tokens of one propensity; the result is a
    tree of tuples: ("num", value), ("comp", p), ("gd", i),
    ("neg", a), (op, a, b)."""

    def __init__(self, toks, comps, gnames):
        self.t, self.i, self.comps, self.gnames = toks, 0, comps, gnames

    def peek(self):
        return self.t[self.i] if self.i < len(self.t) else (None, None)

    def take(self):
        tok = self.peek()
        self.i += 1
        return tok

    def parse(self):
        e = self.sum()
        if self.i != len(self.t):
            raise ParseError(f"unexpected {self.peek()[1]!r}")
        return e

    def sum(self):
        e = self.product()
        while self.peek() in (("op", "+"), ("op", "-")):
            op = self.take()[1]
            e = (op, e, self.product())
        return e

    def product(self):
        e = self.unary()
        while self.peek() in (("op", "*"), ("op", "/")):
            op = self.take()[1]
            e = (op, e, self.unary())
        return e

    def unary(self):
        if self.peek() == ("op", "-"):
            self.take()
            return ("neg", self.unary())
        if self.peek() == ("op", "+"):
            self.take()
            return self.unary()
        return self.primary()

    def primary(self):
        kind, val = self.take()
        if kind == "num":
            return ("num", float(val))
        if kind == "name":
            if val in self.comps:
                return ("comp", self.comps.index(val))
            if val in self.gnames:
                return ("gd", self.gnames.index(val))
            raise ParseError(f"unknown name {val!r}")
        if (kind, val) == ("op", "("):
            e = self.sum()
            if self.take() != ("op", ")"):
                raise ParseError("missing ')'")
            return e
        raise ParseError(f"unexpected {val!r}")


def _side(text, comps):
    counts = np.zeros(len(comps), dtype=np.int64)
    text = text.strip()
    if text == "@":
        return counts
    for term in text.split("+"):
        term = term.strip()
        m = re.fullmatch(r"(?:(\d+)\s*\*\s*)?([A-Za-z_.][A-Za-z0-9_.]*)", term)
        if not m or m.group(2) not in comps:
            raise ParseError(f"bad compartment term {term!r}")
        counts[comps.index(m.group(2))] += int(m.group(1) or 1)
    return counts


def _reads(e, acc):
    if e[0] == "comp":
        acc.add(e[1])
    elif e[0] == "neg":
        _reads(e[1], acc)
    elif e[0] in "+-*/":
        _reads(e[1], acc)
        _reads(e[2], acc)
    return acc


def _c(e):
    kind = e[0]
    if kind == "num":
        return "(" + float(e[1]).hex() + ")"
    if kind == "comp":
        return f"((double)u[{e[1]}])"
    if kind == "gd":
        return f"gd[{e[1]}]"
    if kind == "neg":
        return f"(-{_c(e[1])})"
    return f"({_c(e[1])} {kind} {_c(e[2])})"


@dataclass
class Parsed:
    compartments: list
    gdata_names: list
    S: np.ndarray      # (n_comp, n_trans) int32
    G: np.ndarray      # (n_trans, n_trans) int32
    trees: list
    c_source: str


def parse(transitions, compartments, gdata_names):
    comps, gnames = list(compartments), list(gdata_names)
    if len(set(comps)) != len(comps) or set(comps) & set(gnames) or "@" in comps:
        raise ParseError("compartment and gdata names must be distinct")
    T = len(transitions)
    S = np.zeros((len(comps), T), dtype=np.int32)
    trees = []
    for j, tr in enumerate(transitions):
        parts = tr.split("->")
        if len(parts) != 3:
            raise ParseError(f"{tr!r}: expected 'LHS -> propensity -> RHS'")
        S[:, j] = _side(parts[2], comps) - _side(parts[0], comps)
        trees.append(_Expr(_tokens(parts[1]), comps, gnames).parse())
    G = np.zeros((T, T), dtype=np.int32)
    for k, e in enumerate(trees):
        reads = _reads(e, set())
        for j in range(T):
            if any(S[p, j] != 0 for p in reads):
                G[k, j] = 1
    lines = ["double sg_oracle_rate(int j, const int *u, const double *gd)", "{",
             "    (void)u; (void)gd;", "    switch (j) {"]
    for j, e in enumerate(trees):
        lines.append(f"    case {j}: return {_c(e)};")
    lines += ["    }", "    return 0.0;", "}", ""]
    return Parsed(comps, gnames, S, G, trees, "\n".join(lines))


class _Compiled:
    def __init__(self, path, parsed):
        self.parsed = parsed
        self.lib = ctypes.CDLL(path)
        fn = self.lib.sg_oracle_rate
        self.address = ctypes.cast(fn, ctypes.c_void_p).value
        fn.argtypes = [ctypes.c_int, ctypes.POINTER(ctypes.c_int),
                       ctypes.POINTER(ctypes.c_double)]
        fn.restype = ctypes.c_double
        self.fn = fn


_cache = {}


def compiled(spec):
    """Parse a model spec (dict with transitions, compartments, gdata_names)
    and compile its propensities with gcc; cached per source."""
    p = spec if isinstance(spec, Parsed) else parse(
        spec["transitions"], spec["compartments"], spec["gdata_names"])
    key = hashlib.sha1(p.c_source.encode()).hexdigest()[:16]
    if key not in _cache:
        os.makedirs(_BUILD, exist_ok=True)
        src = os.path.join(_BUILD, f"mparse_{key}.c")
        lib = os.path.join(_BUILD, f"mparse_{key}.so")
        if not os.path.exists(lib):
            with open(src, "w") as f:
                f.write(p.c_source)
            tmp = lib + f".tmp{os.getpid()}"
            subprocess.run(["gcc", "-O2", "-std=c99", "-ffp-contract=off", "-fno-fast-math",
                            "-fPIC", "-shared", "-o", tmp, src], check=True)
            os.replace(tmp, lib)
        _cache[key] = _Compiled(lib, p)
    return _cache[key]


def evaluate(tree, u, gd):
    """Plain Python evaluation of a propensity tree (same grouping)."""
    kind = tree[0]
    if kind == "num":
        return tree[1]
    if kind == "comp":
        return float(u[tree[1]])
    if kind == "gd":
        return float(gd[tree[1]])
    if kind == "neg":
        return -evaluate(tree[1], u, gd)
    a, b = np.float64(evaluate(tree[1], u, gd)), np.float64(evaluate(tree[2], u, gd))
    with np.errstate(all="ignore"):
        return float({"+": a + b, "-": a - b, "*": a * b, "/": a / b}[kind])
