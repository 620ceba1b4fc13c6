"""The oracle's pins must catch plausible mistakes.  Each case copies
oracle/rcg_oracle.c, plants one mistake in the copy (a dropped term, a wrong
index or sign, a transposed operand), builds it on the CPU and runs the pin
suite against it; the suite has to fail."""
import os
import subprocess
import sys
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "rcg_oracle.c")

MUTANTS = {
    "f_without_constant_term": ("return (((u128)1) << p) - 1;", "return (((u128)1) << p) - 2;"),
    "carry_instead_of_xor": ("r ^= a << sh;", "r |= a << sh;"),
    "rows_reversed": ("a |= (u64)((row[b >> 3] >> (b & 7)) & 1u) << r;",
                      "a |= (u64)((row[b >> 3] >> (b & 7)) & 1u) << (L->rows - 1 - r);"),
    "q_weight_off_by_one": ("Q ^= oracle_ring_mul(p, g[k], d);", "Q ^= oracle_ring_mul(p, g[k + 1], d);"),
    "p_drops_a_term": ("                P ^= d;\n", "                P ^= (k ? d : 0);\n"),
    "dd_wrong_weight": ("rhs ^= oracle_ring_mul(p, g[k] ^ g[i], d[k]);", "rhs ^= oracle_ring_mul(p, g[k] ^ g[j], d[k]);"),
    "dd_transposed_solve": ("rhs = oracle_ring_mul(p, g[i], P) ^ Q;", "rhs = oracle_ring_mul(p, g[j], P) ^ Q;"),
    "dd_back_substitution_dropped": ("u64 di = P ^ d[j];", "u64 di = P;"),
    "dp_missing_inverse": ("d[i] = oracle_ring_mul(p, gi_inv, acc);", "d[i] = oracle_ring_mul(p, g[i], acc);"),
    "dq_drops_survivors": ("            acc ^= d[k];\n", "            acc ^= 0;\n"),
    "euclid_swapped_cofactors": ("u128 r0 = f, r1, s0 = 0, s1 = 1;", "u128 r0 = f, r1, s0 = 1, s1 = 0;"),
    "degraded_read_drops_p": ("for (unsigned k = 0; k <= N; k++)", "for (unsigned k = 0; k < N; k++)"),
    "qext_weight_exponent_off_by_one": ("return 1u ^ oracle_ring_xpow(p, k - p + 1);",
                                        "return 1u ^ oracle_ring_xpow(p, k - p);"),
    "qext_weight_drops_identity": ("return 1u ^ oracle_ring_xpow(p, k - p + 1);", "return oracle_ring_xpow(p, k - p + 1);"),
    "cone_check_ignores_common_factor": ("if (poly_gcd(xp1, t) != 1)", "if (poly_gcd(xp1, t) == 0)"),
    "ord2_counts_from_zero": ("unsigned d = 1, v = 2 % p;", "unsigned d = 0, v = 2 % p;"),
    "extension_allowed_for_every_prime": ("if (N > p && !oracle_cone_extends(p))", "if (N > p && 0)"),
    "update_wrong_stripe": ("return oracle_encode(p, N, C, buf + stripe * stripe_stride, 1,",
                            "return oracle_encode(p, N, C, buf, 1,"),
    "h_bits_reversed": ("a |= (u64)((strip[t >> 3] >> (t & 7)) & 1u) << r;",
                        "a |= (u64)((strip[t >> 3] >> (t & 7)) & 1u) << (L->rows - 1 - r);"),
    "h_scatter_toggles": ("if ((a >> r) & 1u)\n                strip[t >> 3] |= m;",
                          "if ((a >> r) & 1u)\n                strip[t >> 3] ^= m;"),
    "h_element_stride": ("const uint8_t *strip = L->base + s * L->stripe_stride + (u64)k * L->strip_stride;\n"
                         "        for (unsigned r = 0; r < L->rows; r++) {\n            u64 t = b * L->rows + r;",
                         "const uint8_t *strip = L->base + s * L->stripe_stride + (u64)k * L->strip_stride;\n"
                         "        for (unsigned r = 0; r < L->rows; r++) {\n            u64 t = b * (L->rows + 1) + r;"),
    # the coefficient-array path for large primes (Z_257)
    "big_mul_drops_top_term": ("        for (int j = 0; j <= b->deg; j++)\n            r.c[i + j] ^= b->c[j];",
                               "        for (int j = 0; j < b->deg; j++)\n            r.c[i + j] ^= b->c[j];"),
    "big_f_one_term_short": ("    for (unsigned t = 0; t < p; t++)\n        f->c[t] = 1;",
                             "    for (unsigned t = 1; t < p; t++)\n        f->c[t] = 1;"),
    "big_euclid_swapped_cofactors": ("    s1.c[0] = 1;\n    s1.deg = 0;", "    s0.c[0] = 1;\n    s0.deg = 0;"),
    "big_weight_off_by_one": ("    bp_xpow(p, k, out);\n}", "    bp_xpow(p, k + 1, out);\n}"),
    "big_gather_element_stride": ("        const u64 t = e * (p - 1) + r;\n        a->c[r]",
                                  "        const u64 t = e * p + r;\n        a->c[r]"),
    "big_dd_wrong_cofactor": ("bp_add(&g[k], &g[a], &w);", "bp_add(&g[k], &g[b], &w);"),
    "big_dp_without_inverse": ("bp_ring_mul(p, &inv, &acc, &da);", "da = acc;"),
    "big_dq_forgets_p": ("bp_gather(p, buf, ss, st, s, N, e, &da);", "bp_zero(&da);"),
}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, "mutation site not found: " + name
    with tempfile.TemporaryDirectory() as d:
        mutant = os.path.join(d, "rcg_oracle_mutant.c")
        so = os.path.join(d, "librcg_oracle_mutant.so")
        open(mutant, "w").write(src.replace(old, new))
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-shared", "-fPIC", "-o", so, mutant])
        env = dict(os.environ, RCG_ORACLE_LIB=so)
        r = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                            os.path.join(ROOT, "tests", "test_oracle_pins.py"),
                            os.path.join(ROOT, "tests", "test_oracle_qext_pins.py"),
                            os.path.join(ROOT, "tests", "test_oracle_horizontal_pins.py"),
                            os.path.join(ROOT, "tests", "test_oracle_p257_pins.py")],
                           cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
        assert r.returncode != 0, "planted mistake %r passed every pin:\n%s" % (name, r.stdout[-2000:])
