"""Oracle vs hand-derived bitstreams (tests/golden/*.txt).

Each fixture's words were derived by hand from the paper's definitions; they pin
the field layout and the bit order of Listing 2 (Section 3.7.2), independent of
the oracle's own code.
"""
import os

import numpy as np
import pytest

import oracle
from helpers import csr_from_edges, parse_golden, words_to_int

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
MODES = {"global": oracle.ID_GLOBAL, "local": oracle.ID_LOCAL, "local_gap": oracle.ID_LOCAL_GAP}


def _fixtures():
    return sorted(f for f in os.listdir(GOLDEN) if f.endswith(".txt"))


def _graph(fx):
    g = fx["graph"]
    return csr_from_edges(g["n"], g["edges"], g.get("weights"))


@pytest.mark.parametrize("name", _fixtures())
def test_golden_streams(name):
    fx = parse_golden(os.path.join(GOLDEN, name))
    n = fx["graph"]["n"]
    rp, col, wt = _graph(fx)
    # relabeled fixtures: DM ([relabel]) or the greedy heuristic ([greedy_relabel])
    rsec = "greedy_relabel" if "greedy_relabel" in fx else ("relabel" if "relabel" in fx else None)
    relabel = {"relabel": oracle.RELABEL_DM, "greedy_relabel": oracle.RELABEL_GREEDY, None: 0}[rsec]
    checked = 0
    for sec, mode in MODES.items():
        if sec not in fx:
            continue
        exp = fx[sec]
        for off in (oracle.OFF_PACKED, oracle.OFF_EF):
            e = oracle.encode(n, rp, col, wt, id_mode=mode, off_mode=off, relabel=relabel, sample=512)
            assert e.bits_A == exp["bits_A"]
            assert words_to_int(e.A, e.bits_A + 64) == exp["A"], f"{sec}: A stream"
            assert list(e.x) == exp["x"]
            for k in ("s", "H", "omega"):
                if k in exp:
                    assert getattr(e, k) == exp[k], k
            if off == oracle.OFF_PACKED and "O" in exp:
                assert e.w_O == exp["w_O"]
                assert words_to_int(e.O, (n + 1) * e.w_O + 64) == exp["O"]
            if off == oracle.OFF_EF and "ef_high" in exp:
                assert e.ef_l == exp["ef_l"]
                assert e.ef_high_bits == exp["ef_high_bits"]
                assert words_to_int(e.ef_high, e.ef_high_bits + 64) == exp["ef_high"]
                assert words_to_int(e.ef_low, e.ef_low_bits + 64) == exp.get("ef_low", 0)
                if "samples" in exp:
                    assert int(e.samples[0]) == exp["samples"]
            if relabel:
                assert list(e.perm) == fx[rsec]["perm"]
                assert list(e.inv_perm) == fx[rsec]["inv_perm"]
            # padding and guard words are zero
            used = (e.bits_A + 63) // 64
            assert not np.any(e.A[used:])
            checked += 1
    assert checked >= 2
