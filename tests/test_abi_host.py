"""CPU-only checks of the C ABI library: it loads, exports every function that
include/rpq.h declares, and its host-side regex compiler produces exactly the
oracle's minimal DFA (canonical numbering makes the tables comparable)."""

import os
import re

import numpy as np
import pytest

import oracle
from paper_2602_20748_gb300 import synth
from conftest import ROOT

rpq = pytest.importorskip("paper_2602_20748_gb300.rpq")


def header_functions():
    text = open(os.path.join(ROOT, "include", "rpq.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"^\s*(?:const\s+)?\w+\s*\**\s*(\w+)\s*\(", text, flags=re.M)))


def test_library_exports_every_declared_function():
    names = header_functions()
    assert len(names) >= 17
    for name in names:
        assert hasattr(rpq._lib, name), name
    assert sorted(rpq.EXPORTED) == names


@pytest.fixture(scope="module")
def hctx():
    return rpq.Context(device=-1)


def gpu_dfa(hctx, regex, names=None):
    q = rpq.compile_rpq(hctx, regex, names)
    return rpq.query_info(q)


PAPER_QUERIES = ["a*", "a?b*", "ab*", "abcd", "abc*", "ab*c", "(a|b|c)b*", "a*b*", "ab*c*", "(a|b|c)*"]
CONFIG_QUERIES = ["a.b.c*", "a*", "(a|b)+·c", "a·b*·c", "(a·b)*", "b.c*", "d*"]


@pytest.mark.parametrize("regex", PAPER_QUERIES + CONFIG_QUERIES)
def test_compiler_matches_oracle_dfa(hctx, regex):
    ns, fmask, nxt = gpu_dfa(hctx, regex)
    L = nxt.shape[1]
    k, fin, onxt = oracle.dfa(regex, L)
    assert ns == k
    assert [bool(fmask >> q & 1) for q in range(ns)] == fin.tolist()
    assert nxt.tolist() == onxt.tolist()


@pytest.mark.parametrize("case", range(300))
def test_compiler_random_regexes(hctx, case):
    regex = synth.random_regex(40_000 + case, 1 + case % 6, max_symbols=6)
    ns, fmask, nxt = gpu_dfa(hctx, regex)
    L = nxt.shape[1] if ns else 1
    k, fin, onxt = oracle.dfa(regex, L)
    assert ns == k, regex
    if ns:
        assert [bool(fmask >> q & 1) for q in range(ns)] == fin.tolist()
        assert nxt.tolist() == onxt.tolist(), regex


def test_compiler_named_labels(hctx):
    names = ["knows", "likes", "replyOf"]
    ns, fmask, nxt = gpu_dfa(hctx, "knows.replyOf*", names)
    assert ns == 2 and nxt.shape[1] == 3
    with pytest.raises(rpq.RPQError) as e:
        gpu_dfa(hctx, "hates", names)
    assert e.value.code == rpq.RPQ_ERR_UNKNOWN_LABEL


@pytest.mark.parametrize("bad", ["a|", "(a", "*a", "a)", "", "a**(", "A", "a..b", "()"])
def test_parse_errors(hctx, bad):
    with pytest.raises(rpq.RPQError) as e:
        gpu_dfa(hctx, bad)
    assert e.value.code == rpq.RPQ_ERR_PARSE
    with pytest.raises(oracle.OracleError):
        oracle.dfa(bad, 2)


def test_too_complex(hctx):
    # (a|b)* a (a|b)^5: the minimal DFA needs 2^6 = 64 states
    with pytest.raises(rpq.RPQError) as e:
        gpu_dfa(hctx, "(a|b)*a(a|b)(a|b)(a|b)(a|b)(a|b)")
    assert e.value.code == rpq.RPQ_ERR_TOO_COMPLEX
    with pytest.raises(rpq.RPQError) as e:
        gpu_dfa(hctx, "a" * 64)
    assert e.value.code == rpq.RPQ_ERR_TOO_COMPLEX
    ns, _, _ = gpu_dfa(hctx, "(a|b)*a(a|b)(a|b)(a|b)(a|b)")  # 32 states: at the limit
    assert ns == 32


def test_host_only_context_refuses_device_work(hctx):
    with pytest.raises(rpq.RPQError) as e:
        rpq.load_graph(hctx, 2, 1, [0], [1], [0])
    assert e.value.code == rpq.RPQ_ERR_NO_DEVICE


def test_device_context_fails_loudly_without_gpu():
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(rpq.RPQError) as e:
        rpq.Context(device=0)
    assert e.value.code == rpq.RPQ_ERR_CUDA


def test_options_round_trip(hctx):
    rpq.rpq_set_option(hctx, "alpha", 8)
    assert rpq.rpq_get_option(hctx, "alpha") == 8
    rpq.rpq_set_option(hctx, "batch_evict", 4096)
    assert rpq.rpq_get_option(hctx, "batch_evict") == 4096
    assert rpq.rpq_get_option(hctx, "batch_threads") in (128, 256, 512)
    with pytest.raises(rpq.RPQError):
        rpq.rpq_get_option(hctx, "no_such_option")
    rpq.rpq_set_option(hctx, "alpha", 16)


def test_stream_open_multi_argument_checks(hctx):
    """rpq_stream_open_multi validates its arguments before touching the graph
    or the device: no queries or a null query is INVALID_ARG, a host-only
    context is NO_DEVICE (the graph handle is never read on these paths)."""
    import ctypes

    q = rpq.compile_rpq(hctx, "a*")
    out = ctypes.c_void_p()
    fake_graph = ctypes.c_void_p(1)  # never dereferenced on the paths below
    one = (ctypes.c_void_p * 1)(q.h)
    none = (ctypes.c_void_p * 1)(None)
    f = rpq._lib.rpq_stream_open_multi
    assert f(hctx.h, None, one, 1, 0, 0, 0, ctypes.byref(out)) == rpq.RPQ_ERR_INVALID_ARG
    assert f(hctx.h, fake_graph, one, 0, 0, 0, 0, ctypes.byref(out)) == rpq.RPQ_ERR_INVALID_ARG
    assert f(hctx.h, fake_graph, none, 1, 0, 0, 0, ctypes.byref(out)) == rpq.RPQ_ERR_INVALID_ARG
    assert f(hctx.h, fake_graph, one, 1, 0, 0, 0, ctypes.byref(out)) == rpq.RPQ_ERR_NO_DEVICE
    assert out.value is None
