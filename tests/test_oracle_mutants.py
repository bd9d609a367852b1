"""The oracle's pins are sensitive: a plausible mistake planted anywhere in a
copy of the oracle (a dropped term, a wrong sign or index, a swapped
operand, a wrong constant) makes the pin suite fail.  Each mutant is a text
substitution in oracle/bicoptor_oracle.c, built into a temporary directory
and run against tests/test_oracle_pins.py in a subprocess; the mutants'
subprocesses run side by side."""
import concurrent.futures as cf
import os
import subprocess
import sys

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(ROOT, "oracle", "bicoptor_oracle.c")

MUTANTS = {
    "cut_keeps_weights": ("out |= bit << (i - k1);", "out |= bit << i;"),
    "p1_trunc_no_negation": ("return rneg(orc_cut(a, ell, k1, k2), ell - k1 - k2);",
                             "return rmod(orc_cut(a, ell, k1, k2), ell - k1 - k2);"),
    "newtrc2_k1_k2_swapped": ("return rmod(orc_cut(s0, ell, k1, k2), ell - k1 - k2);",
                              "return rmod(orc_cut(s0, ell, k2, k1), ell - k1 - k2);"),
    "step4_dropped_minus_one": ("v0[i] = rmod(u0[i] + u0[i + 1] - 1, lx);",
                                "v0[i] = rmod(u0[i] + u0[i + 1], lx);"),
    "step4_wrong_neighbour": ("v1[i] = rmod(u1[i] + u1[i + 1], lx);",
                              "v1[i] = rmod(u1[i] + u1[i], lx);"),
    "modswitch_p1_dropped_term": ("return (uint32_t)(((uint64_t)p + b - pow2) % p);",
                                  "return (uint32_t)(((uint64_t)p + b) % p);"),
    "reshare_wrong_sign": ("msg1[k] = (uint32_t)(((uint64_t)sh1[k] + p - z[k]) % p);",
                           "msg1[k] = (uint32_t)(((uint64_t)sh1[k] + z[k]) % p);"),
    "flip_inverted": ("if (t) { s0 = rneg(s0, ell); s1 = rneg(s1, ell); }",
                      "if (!t) { s0 = rneg(s0, ell); s1 = rneg(s1, ell); }"),
    "shuffle_off_by_one": ("int partner = (int)(((uint64_t)W * (uint64_t)(j + 1)) >> 32);",
                           "int partner = (int)(((uint64_t)W * (uint64_t)j) >> 32);"),
    "beaver_dropped_de": ("o0[i] = rmod(d * e + d * T.b0 + e * T.a0 + T.c0, ell);",
                          "o0[i] = rmod(d * T.b0 + e * T.a0 + T.c0, ell);"),
    "relu_unflip_dropped_t_x": ("o0[i] = rmod((uint64_t)t * s0[i] + one_m2t * xd0, ell);",
                                "o0[i] = rmod(one_m2t * xd0, ell);"),
    "philox_wrong_multiplier": ("#define PHILOX_M0 0xD2511F53u", "#define PHILOX_M0 0xD2511F55u"),
    "philox_key_bump_order": ("if (round > 0) { k0 += PHILOX_W0; k1 += PHILOX_W1; }",
                              "{ k0 += PHILOX_W0; k1 += PHILOX_W1; }"),
    "share_sign": ("*s1 = rneg(r, ell);", "*s1 = rmod(r, ell);"),
    "rss_xor_dropped_product": ("X[j] = rmod(S[j] + T[j] - 2 * ST[j], ell);",
                                "X[j] = rmod(S[j] + T[j], ell);"),
    "rss_zero_sharing_sign": ("out[i] = rmod(a[i] * b[i] + a[i] * b[j] + a[j] * b[i] + g[i] - g[j], ell);",
                              "out[i] = rmod(a[i] * b[i] + a[i] * b[j] + a[j] * b[i] + g[i] + g[j], ell);"),
    "mask_skipped_for_p1": ("sh1[k] = (uint32_t)(((uint64_t)sh1[k] * r[k]) % p);",
                            "sh1[k] = sh1[k];"),
    "mask_rho_can_be_zero": ("uint32_t rho = 1u + (uint32_t)(((u128)wr * (u128)(P->p - 1u)) >> 64);",
                             "uint32_t rho = (uint32_t)(((u128)wr * (u128)(P->p - 1u)) >> 64);"),
    "shuffle_p0_only": ("sh0[k] = m0[perm[k]]; sh1[k] = m1[perm[k]];",
                        "sh0[k] = m0[perm[k]]; sh1[k] = m1[k];"),
    "trunc_then_mul_y_by_kx": ("uint64_t ty0 = smltrc_p0(y0[i], ell, ky), ty1 = smltrc_p1(y1[i], ell, ky);",
                               "uint64_t ty0 = smltrc_p0(y0[i], ell, kx), ty1 = smltrc_p1(y1[i], ell, kx);"),
    "aby3_signed_division": ("if (ell < 128 && (v >> (ell - 1)) & 1) v -= ((__int128)1 << ell);",
                             "if (0) v -= ((__int128)1 << ell);"),
    # the per-element draws of Alg. drelu / Alg. relu from the Philox streams
    "z_draw_modulus_p_minus_1": ("z[k] = (uint32_t)(((u128)wz * (u128)P->p) >> 64);",
                                 "z[k] = (uint32_t)(((u128)wz * (u128)(P->p - 1u)) >> 64);"),
    "mask_without_two_inv32": ("r[k] = (uint32_t)(((uint64_t)rho * inv32) % P->p);",
                               "r[k] = rho % P->p;"),
    "mask_words_swapped": ("uint64_t wr = (uint64_t)orc_stream_word(seed, PAIR_01, PUR_MASK, tid, elem, 4 * k) |",
                           "uint64_t wr = (uint64_t)orc_stream_word(seed, PAIR_01, PUR_MASK, tid, elem, 4 * k + 2) |"),
    "reply_from_seed12": ("msg1);\n        uint64_t d0 = stream_ring(seed, PAIR_02, PUR_REPLY, tid, elem, 0, ell);",
                          "msg1);\n        uint64_t d0 = stream_ring(seed, PAIR_12, PUR_REPLY, tid, elem, 0, ell);"),
    "triple_b0_is_c0": ("T.b0 = stream_ring(seed, PAIR_02, purpose, tid, elem, 1, ell);",
                        "T.b0 = stream_ring(seed, PAIR_02, purpose, tid, elem, 2, ell);"),
    "ring_draw_high_word_first": ("return rmod(lo | (hi << 32), ell);",
                                  "return rmod(hi | (lo << 32), ell);"),
    "shuffle_words_reversed": ("uint32_t W = fy[lx - j + 1];", "uint32_t W = fy[j];"),
    "mul_triple_relu_purpose": ("triple_t T = draw_triple(seed, PUR_MUL_TRIPLE, tid, elem_index(idx, i), ell);",
                                "triple_t T = draw_triple(seed, PUR_RELU_TRIPLE, tid, elem_index(idx, i), ell);"),
    "rss_alpha_from_seed01": ("for (int j = 0; j < 3; j++) al[j] = stream_ring(seed, PAIR_012, PUR_RSS_T, tid, elem, j, ell);",
                              "for (int j = 0; j < 3; j++) al[j] = stream_ring(seed, PAIR_01, PUR_RSS_T, tid, elem, j, ell);"),
    "rss_s_from_seed012": ("uint64_t sbit = orc_stream_word(seed, PAIR_2, PUR_RSS_S, tid, elem, 0) & 1u;",
                           "uint64_t sbit = orc_stream_word(seed, PAIR_012, PUR_RSS_S, tid, elem, 0) & 1u;"),
    "rss_relu_reuses_gamma": ("gr[j] = stream_ring(seed, PAIR_012, PUR_RSS_ZR, tid, elem, j, ell);",
                              "gr[j] = stream_ring(seed, PAIR_012, PUR_RSS_Z, tid, elem, j, ell);"),
    "aby3_rp0_is_r0": ("uint64_t rp0 = stream_ring(seed, PAIR_02, PUR_ABY3, tid, elem, 1, ell);",
                       "uint64_t rp0 = stream_ring(seed, PAIR_02, PUR_ABY3, tid, elem, 0, ell);"),
    "aby3_r1_from_seed02": ("uint64_t r1 = stream_ring(seed, PAIR_12, PUR_ABY3, tid, elem, 0, ell);",
                            "uint64_t r1 = stream_ring(seed, PAIR_02, PUR_ABY3, tid, elem, 2, ell);"),
    "dealer_from_seed01": ("uint64_t R = stream_ring(seed, PAIR_DEALER, PUR_SHARE, tid, elem_index(idx, i), 0, ell);",
                           "uint64_t R = stream_ring(seed, PAIR_01, PUR_SHARE, tid, elem_index(idx, i), 0, ell);"),
    # the Bicoptor 1.0-style protocol
    "b1_sums_not_recursive": ("acc0 = rmod(acc0 + u0[i], ell);", "acc0 = rmod(u0[i], ell);"),
    "b1_p0_constant_dropped": ("v0[i] = rmod(acc0 - 1, ell);", "v0[i] = acc0;"),
    "b1_mask_may_be_even": ("r[k] = rmod(wr | 1u, P->ell);", "r[k] = rmod(wr, P->ell);"),
    "b1_reshare_wrong_sign": ("msg1[k] = rmod(sh1[k] * r[k] - z[k], ell);",
                              "msg1[k] = rmod(sh1[k] * r[k] + z[k], ell);"),
    "b1_trunc_in_small_ring": ("u1[i] = smltrc_p1(s1, ell, c + i);",
                               "u1[i] = rmod(smltrc_p1(s1, ell, c + i), lx);"),
}


def _run_mutant(name, workdir):
    """Build the oracle with mutant `name` planted and run the pin suite on
    it; returns (pytest exit code, its stdout)."""
    old, new = MUTANTS[name]
    src = open(SRC).read()
    if src.count(old) != 1:
        return None, f"mutant {name} no longer matches the oracle source"
    mutant = os.path.join(workdir, "bicoptor_oracle.c")
    with open(mutant, "w") as f:
        f.write(src.replace(old, new))
    # the pin suites of the mutants run side by side, two OpenMP threads each
    env = dict(os.environ, BICOPTOR_ORACLE_SRC=mutant, PYTHONPATH=ROOT, OMP_NUM_THREADS="2")
    proc = subprocess.run([sys.executable, "-m", "pytest", "-x", "-q", "-p", "no:cacheprovider",
                           os.path.join(HERE, "test_oracle_pins.py")],
                          cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    return proc.returncode, proc.stdout


@pytest.fixture(scope="module")
def mutant_runs(request, tmp_path_factory):
    """The pin-suite runs of every mutant selected in this session, made
    concurrently (each in its own directory and process)."""
    names = sorted({it.callspec.params["name"] for it in request.session.items
                    if getattr(it, "originalname", "") == "test_pins_catch_planted_mistake"})
    dirs = {n: str(tmp_path_factory.mktemp(f"mutant_{n}")) for n in names}
    workers = max(1, min(len(names), (os.cpu_count() or 2) // 2))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        futs = {n: ex.submit(_run_mutant, n, dirs[n]) for n in names}
        return {n: f.result() for n, f in futs.items()}


@pytest.mark.slow
@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_planted_mistake(name, mutant_runs):
    rc, out = mutant_runs[name]
    assert rc is not None, out
    assert rc != 0, f"no pin caught mutant {name}:\n{out[-1500:]}"
    assert "failed" in out or "error" in out.lower()
