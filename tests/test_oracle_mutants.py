"""Plant plausible mistakes in a copy of the oracle (CPU only) and check that
at least one pin catches each: evidence that the pins can tell a wrong
oracle from a right one.  Every mutant keeps all memory accesses in bounds."""
import pytest

import oracle
import oracle_pins as P

MUTANTS = [
    ("philox: wrong product word", "uint32_t y0 = hi1 ^ x1 ^ k0;", "uint32_t y0 = hi0 ^ x1 ^ k0;"),
    ("philox: key not bumped", "    k1 += W1;\n", "\n"),
    ("naive: last neighbour never drawn",
     "const uint64_t x = uniform_below(B, (uint64_t)d);\n        next = g->col[off + (int64_t)x];",
     "const uint64_t x = uniform_below(B, (uint64_t)(d > 1 ? d - 1 : d));\n        next = g->col[off + (int64_t)x];"),
    ("alias: donor loses the wrong mass", "q[l] -= S - q[s];", "q[l] -= q[s];"),
    ("alias: probability scaled by 2^31", "(((unsigned __int128)q[s] << 32) / S)", "(((unsigned __int128)q[s] << 31) / S)"),
    ("alias: first and second swapped in generation", "(y < g->H[off + x])", "(y >= g->H[off + x])"),
    ("threshold: ceiling instead of floor", "return (uint64_t)floor(t * 4294967296.0);",
     "return (uint64_t)ceil(t * 4294967296.0);"),
    ("quantise: floor instead of round-half-even", "double t = rint((double)w * 65536.0);",
     "double t = floor((double)w * 65536.0);"),
    ("ppr: no stop coin at the source", "if (p->algo == ORC_PPR && (uint64_t)B[3] < T_stop)",
     "if (p->algo == ORC_PPR && s > 0 && (uint64_t)B[3] < T_stop)"),
    ("ppr: stop probability complemented", "const uint64_t T_stop = orc_threshold(p->ppr_stop);",
     "const uint64_t T_stop = orc_threshold(1.0 - p->ppr_stop);"),
    ("metapath: schema index off by one", "p->schema[s % p->schema_len]", "p->schema[(s + 1) % p->schema_len]"),
    ("metapath: CDF search takes <=", "if (x < cdf[mid]) hi = mid;", "if (x <= cdf[mid]) hi = mid;"),
    ("node2vec: return edge gets the far weight", "T = T_ret;", "T = T_far;"),
    ("node2vec: IsNeighbor direction reversed", "is_neighbor(g, c, u, sec)", "is_neighbor(g, u, c, sec)"),
    ("node2vec: prev taken as cur", "const int32_t u = path[s - 1];", "const int32_t u = path[s];"),
    ("node2vec: p* ignores 1/a", "pstar = w_ret > w_nb ? w_ret : w_nb;", "pstar = w_nb;"),
    ("walk: one move short", "if (s == max_len) {", "if (s + 1 == max_len) {"),
]


@pytest.mark.parametrize("name,old,new", MUTANTS, ids=[m[0] for m in MUTANTS])
def test_pins_catch_planted_mistake(name, old, new, tmp_path):
    src = oracle.source_text()
    assert src.count(old) == 1, f"mutation anchor not unique for {name!r}"
    lib = oracle.compile_variant(src.replace(old, new), str(tmp_path), "mutant")
    caught = []
    for pin in P.ALL_PINS:
        try:
            pin(lib)
        except AssertionError:
            caught.append(pin.__name__)
            break
    assert caught, f"no pin caught the planted mistake: {name}"
