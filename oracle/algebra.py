"""Brute-force RPQ evaluation by boolean-matrix algebra.

TEST INFRASTRUCTURE ONLY: a second, independent way to compute Definition 1
(Section 2.1) on small graphs, used to pin the product-BFS oracle.  It follows
the algebra-based approach of Section 2.2: a label is its edge relation,
concatenation is a join (boolean matrix product), alternation is a union, and
a Kleene star is the reflexive transitive closure computed by joining until
no new pair appears (the alpha-operator fixpoint).  No automaton is involved.

    R(l)       = A_l                  (adjacency of label l)
    R(e1 e2)   = R(e1) o R(e2)
    R(e1 | e2) = R(e1) v R(e2)
    R(e*)      = I v R(e)^+
    R(e+)      = R(e)^+
    R(e?)      = I v R(e)

Graphs up to a few thousand vertices.
"""

from __future__ import annotations

import numpy as np

__all__ = ["parse", "relation", "rpq_pairs", "ParseError"]


class ParseError(ValueError):
    pass


def _tokenize(text: str, names):
    toks = []
    i = 0
    while i < len(text):
        c = text[i]
        if c in " \t":
            i += 1
        elif c in "|*+?()":
            toks.append(c)
            i += 1
        elif c == "." or c == "·":
            toks.append(".")
            i += 1
        elif names is None and "a" <= c <= "z":
            toks.append(("L", ord(c) - ord("a")))
            i += 1
        elif names is not None and (c.isalnum() or c == "_"):
            j = i
            while j < len(text) and (text[j].isalnum() or text[j] == "_"):
                j += 1
            ident = text[i:j]
            if ident not in names:
                raise ParseError(f"unknown label {ident!r}")
            toks.append(("L", names.index(ident)))
            i = j
        else:
            raise ParseError(f"unexpected character {c!r} at {i}")
    return toks


def parse(text: str, names=None):
    """Returns a nested tuple tree: ('L', l) | ('cat', a, b) | ('alt', a, b) |
    ('star', a) | ('plus', a) | ('opt', a)."""
    toks = _tokenize(text, names)
    pos = [0]

    def peek():
        return toks[pos[0]] if pos[0] < len(toks) else None

    def take():
        t = peek()
        pos[0] += 1
        return t

    def alt():
        node = cat()
        while peek() == "|":
            take()
            node = ("alt", node, cat())
        return node

    def starts_atom(t):
        return t == "(" or isinstance(t, tuple)

    def cat():
        node = postfix()
        while True:
            t = peek()
            if t == ".":
                take()
                node = ("cat", node, postfix())
            elif starts_atom(t):
                node = ("cat", node, postfix())
            else:
                return node

    def postfix():
        node = atom()
        while peek() in ("*", "+", "?"):
            op = take()
            node = ({"*": "star", "+": "plus", "?": "opt"}[op], node)
        return node

    def atom():
        t = take()
        if t == "(":
            node = alt()
            if take() != ")":
                raise ParseError("expected ')'")
            return node
        if isinstance(t, tuple):
            return t
        raise ParseError(f"unexpected token {t!r}")

    tree = alt()
    if peek() is not None:
        raise ParseError("trailing tokens")
    return tree


def _join(x: np.ndarray, y: np.ndarray) -> np.ndarray:
    # Boolean product through an exact float64 matrix product (counts < 2^53).
    return (x.astype(np.float64) @ y.astype(np.float64)) > 0


def _closure_plus(x: np.ndarray) -> np.ndarray:
    """R^+ : join until a fixpoint (each round doubles the path length)."""
    c = x.copy()
    while True:
        nxt = c | _join(c, c)
        if np.array_equal(nxt, c):
            return c
        c = nxt


def relation(tree, adj: list[np.ndarray], n: int) -> np.ndarray:
    kind = tree[0]
    if kind == "L":
        l = tree[1]
        return adj[l].copy() if l < len(adj) else np.zeros((n, n), dtype=bool)
    if kind == "cat":
        return _join(relation(tree[1], adj, n), relation(tree[2], adj, n))
    if kind == "alt":
        return relation(tree[1], adj, n) | relation(tree[2], adj, n)
    ident = np.eye(n, dtype=bool)
    if kind == "star":
        return ident | _closure_plus(relation(tree[1], adj, n))
    if kind == "plus":
        return _closure_plus(relation(tree[1], adj, n))
    if kind == "opt":
        return ident | relation(tree[1], adj, n)
    raise ValueError(kind)


def adjacency(n: int, n_labels: int, src, dst, label) -> list[np.ndarray]:
    adj = [np.zeros((n, n), dtype=bool) for _ in range(n_labels)]
    for s, d, l in zip(np.asarray(src), np.asarray(dst), np.asarray(label)):
        adj[int(l)][int(s), int(d)] = True
    return adj


def rpq_pairs(n: int, n_labels: int, src, dst, label, regex: str, names=None) -> np.ndarray:
    """All-pairs result as an (k, 2) uint32 array sorted lexicographically."""
    tree = parse(regex, names)
    r = relation(tree, adjacency(n, n_labels, src, dst, label), n)
    s, d = np.nonzero(r)  # row-major order = lexicographic
    return np.stack([s, d], axis=1).astype(np.uint32)
