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
    ("its: exclusive prefix sums", "acc += (uint64_t)wq;\n      cdf[e] = acc;", "cdf[e] = acc;\n      acc += (uint64_t)wq;"),
    ("its: CDF search takes <=", "if (x < P[mid]) hi = mid;", "if (x <= P[mid]) hi = mid;"),
    ("its: x drawn below the second-last prefix", "const uint64_t x = uniform_below(B, P[d - 1]);",
     "const uint64_t x = uniform_below(B, d > 1 ? P[d - 2] : P[0]);"),
    ("rej: p* of the first neighbour", "pstar = g->pmax[cur];", "pstar = g->pmax[g->col[off]];"),
    ("rej: p* is the smallest weight", "if ((uint32_t)wq > m) m = (uint32_t)wq;",
     "if (e == row_ptr[v] || (uint32_t)wq < m) m = (uint32_t)wq;"),
    ("rej: threshold rounded up", "return ((uint64_t)W << 32) / pstar;",
     "return (((uint64_t)W << 32) + pstar - 1) / pstar;"),
    ("rej: dart reuses the first draw", "if (a > 0) draw_block(seed, w, (uint32_t)s, a, B);\n          if (st) st->attempts++;\n          const int64_t x = (int64_t)uniform_below(B, (uint64_t)d);\n          const uint32_t Wx",
     "if (a > 0) draw_block(seed, w, (uint32_t)s, a > 1 ? a - 1 : a, B);\n          if (st) st->attempts++;\n          const int64_t x = (int64_t)uniform_below(B, (uint64_t)d);\n          const uint32_t Wx"),
    ("o-rej: bound truncated", "return ORC_ERR_INVALID;\n    double t = rint(p->max_weight * 65536.0);",
     "return ORC_ERR_INVALID;\n    double t = floor(p->max_weight * 65536.0 / 2);"),
    ("weighted node2vec: caller's bound truncated", "return ORC_ERR_INVALID;\n      double t = rint(p->max_weight * 65536.0);",
     "return ORC_ERR_INVALID;\n      double t = floor(p->max_weight * 65536.0 / 2);"),
    ("weighted node2vec: weight word shares the class word",
     "if (!((uint64_t)B[3] < orc_rej_threshold(Wx, P))) continue;",
     "if (!((uint64_t)B[2] < orc_rej_threshold(Wx, P))) continue;"),
    ("weighted node2vec: bound of the previous vertex", "          P = g->pmax[cur];\n          if (sec) sec_touch(sec, SEC_PMAX, (int64_t)cur * 4);",
     "          P = g->pmax[s > 0 ? path[s - 1] : cur];\n          if (sec) sec_touch(sec, SEC_PMAX, (int64_t)cur * 4);"),
    ("weighted node2vec: weight test only after the source", "if (p->algo == ORC_NODE2VEC_WEIGHTED) {\n            const uint32_t Wx",
     "if (p->algo == ORC_NODE2VEC_WEIGHTED && s > 0) {\n            const uint32_t Wx"),
    ("custom: update sees the query before the move", "if (update && update(user, (int64_t)w, s, cur, prev, dst, off + x)) break;",
     "if (update && update(user, (int64_t)w, s - 1, prev, prev, dst, off + x)) break;"),
    ("custom: o-rej dart on word 3", "if ((uint64_t)B[2] < orc_rej_threshold(W, max_weight)) { x = c; break; }",
     "if ((uint64_t)B[3] < orc_rej_threshold(W, max_weight)) { x = c; break; }"),
    ("custom: weight sees the previous vertex as cur", "const uint32_t W = weight(user, (int64_t)w, s, cur, prev, g->col[off + c], off + c);",
     "const uint32_t W = weight(user, (int64_t)w, s, prev, prev, g->col[off + c], off + c);"),
    ("zero row: not a dead end for REJ", "if (pstar == 0) { if (st) st->stop_dead++; break; }",
     "if (pstar == 0) pstar = 1;"),
    ("sectors: IsNeighbor probes not counted", "      sec_touch(sec, SEC_COL, m * 4);\n", "\n"),
    ("sectors: range bound one byte short", "for (int64_t b = byte_lo & ~31LL; b < byte_hi; b += 32)",
     "for (int64_t b = byte_lo & ~31LL; b < byte_hi - 1; b += 32)"),
    ("sectors: range start not rounded to its sector", "for (int64_t b = byte_lo & ~31LL; b < byte_hi; b += 32)",
     "for (int64_t b = byte_lo; b < byte_hi; b += 32)"),
    ("sectors: row pair counted as its first offset only",
     "if (sec) { sec_touch(sec, SEC_ROW, (int64_t)cur * 4); sec_touch(sec, SEC_ROW, (int64_t)(cur + 1) * 4); }",
     "if (sec) { sec_touch(sec, SEC_ROW, (int64_t)cur * 4); }"),
    ("sectors: ITS search probes not counted", "          if (sec) sec_touch(sec, SEC_CDF, (off + mid) * 8);\n", "\n"),
    ("sectors: REJ bound not counted", "          if (sec) sec_touch(sec, SEC_PMAX, (int64_t)cur * 4);\n          if (pstar == 0)",
     "          if (pstar == 0)"),
    ("return-only count includes the first move", "if (st && p->algo == ORC_NODE2VEC && s > 0 && (uint64_t)B[2] >=",
     "if (st && p->algo == ORC_NODE2VEC && s >= 0 && (uint64_t)B[2] >="),
    ("return-only count against the lower threshold", "(uint64_t)B[2] >= (T_nb > T_far ? T_nb : T_far))",
     "(uint64_t)B[2] >= (T_nb < T_far ? T_nb : T_far))"),
    ("sectors: set cleared once per walk, not per step", "    path[0] = cur;\n    for (;;) {\n      if (sec) sec->n = 0;\n",
     "    path[0] = cur;\n    if (sec) sec->n = 0;\n    for (;;) {\n"),
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
