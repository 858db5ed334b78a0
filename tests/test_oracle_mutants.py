"""Plant plausible mistakes in copies of the oracle and check the pins catch each one.

Each mutant is the oracle's C source with one edit (a dropped term, a wrong
sign, index or comparison, a swapped operand), compiled on the CPU into a
temporary library. The pin suite must report at least one failure for every
mutant; a mutant that every pin accepts would be a blind spot of the pins.
"""
import os
import subprocess

import pytest

from oracle import build as obuild
from oracle.oracle import Oracle
from tests import oracle_pins

MUTANTS = {
    "idf_drop_plus_one": ("(1.0 + (double)df[t])) + 1.0;", "(1.0 + (double)df[t]));"),
    "idf_unsmoothed": ("log((1.0 + (double)n_docs) / (1.0 + (double)df[t]))",
                       "log((double)n_docs / (1.0 + (double)df[t]))"),
    "weights_ignore_idf": ("(double)counts[e] * (idf ? idf[terms[e]] : 1.0)", "(double)counts[e]"),
    "ref_norm_no_sqrt": ("rnorm[p] = sqrt(rnorm[p]);", "rnorm[p] = rnorm[p];"),
    "ref_weight_one": ("double r = idf ? idf[t] : 1.0;", "double r = 1.0;"),
    "sig_no_doc_norm": ("s[p] / (nrm * rnorm[p])", "s[p] / rnorm[p]"),
    "sig_numerator_squared": ("s[p] += w[e] * (idf ? idf[terms[e]] : 1.0);", "s[p] += w[e] * w[e];"),
    "rank_df_ascending": ("return (x->df < y->df) - (x->df > y->df);", "return (x->df > y->df) - (x->df < y->df);"),
    "rank_tiebreak_desc": ("return (x->t > y->t) - (x->t < y->t);", "return (x->t < y->t) - (x->t > y->t);"),
    "partition_cut_off_by_one": ("int64_t hi = ((int64_t)(p + 1) * n_sel) / k;",
                                 "int64_t hi = ((int64_t)(p + 1) * n_sel + 1) / k;"),
    "region_default_strict": ("(double)r[q].df <= (double)n_docs / 100.0", "(double)r[q].df < (double)n_docs / 100.0"),
    "df1_means_df2": ("if (df[t] == 1) sel[n_sel++] = t;", "if (df[t] == 2) sel[n_sel++] = t;"),
    "cos_dense_no_sqrt": ("return ab / (sqrt(aa) * sqrt(bb));\n}\n\n/* Exact", "return ab / (aa * bb);\n}\n\n/* Exact"),
    "cosine_merge_wrong_advance": ("else if (ti[x] < tj[y]) ++x;", "else if (ti[x] < tj[y]) ++y;"),
    "cosine_norm_uses_other_row": ("for (int64_t y = 0; y < nj; ++y) bb += wj[y] * wj[y];",
                                   "for (int64_t y = 0; y < nj; ++y) bb += wi[y] * wj[y];"),
    "counts_off_by_one": ("counts[out] = (int32_t)(y - x);", "counts[out] = (int32_t)(y - x + 1);"),
    "simhash_tie_to_one": ("if (col[b] > 0) f |= (1ULL << b);", "if (col[b] >= 0) f |= (1ULL << b);"),
    "simhash_bit_order": ("col[b] += ((h >> b) & 1ULL) ? 1 : -1;", "col[b] += ((h >> (63 - b)) & 1ULL) ? 1 : -1;"),
    "simhash_no_minus_one": ("col[b] += ((h >> b) & 1ULL) ? 1 : -1;", "col[b] += ((h >> b) & 1ULL) ? 1 : 0;"),
    "splitmix_shift": ("z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;", "z = (z ^ (z >> 31)) * 0xBF58476D1CE4E5B9ULL;"),
    "term_hash_no_seed": ("orc_splitmix64((uint64_t)(uint32_t)t ^ seed)", "orc_splitmix64((uint64_t)(uint32_t)t)"),
    "grams_no_case_fold": ("if (c >= 'A' && c <= 'Z') return c - 'A';", "if (c >= 'A' && c <= 'Z') return -1;"),
    "grams_base_27": ("grams[out++] = 676 * x + 26 * y + z;", "grams[out++] = 729 * x + 27 * y + z;"),
    "grams_reversed_letters": ("grams[out++] = 676 * x + 26 * y + z;", "grams[out++] = 676 * z + 26 * y + x;"),
    "grams_cross_documents": ("p + 2 < text_offsets[d + 1]; ++p)", "p < text_offsets[d + 1]; ++p)"),
    "grams_last_window_dropped": ("p + 2 < text_offsets[d + 1]; ++p)", "p + 3 < text_offsets[d + 1]; ++p)"),
    "md5_round2_index": ("k = (1 + 5 * i) % 16;", "k = (5 * i) % 16;"),
    "md5_round3_shift": ("{4, 11, 16, 23}", "{4, 11, 16, 22}"),
    "md5_I_no_not": ("f = c ^ (b | ~d);", "f = c ^ (b | d);"),
    "md5_length_in_bytes": ("(uint8_t)(((uint64_t)len * 8u) >> (8 * (pos - (padded - 8))))",
                            "(uint8_t)(((uint64_t)len) >> (8 * (pos - (padded - 8))))"),
    "md5_no_feed_forward": ("state[2] += c;", "state[2] = c;"),
    "sha1_rotate_31": ("c = orc_rotl32(b, 30);", "c = orc_rotl32(b, 31);"),
    "sha1_schedule_index": ("W[t - 3] ^ W[t - 8] ^ W[t - 14] ^ W[t - 16]", "W[t - 3] ^ W[t - 8] ^ W[t - 14] ^ W[t - 15]"),
    "sha1_maj_dropped_term": ("f = (b & c) ^ (b & d) ^ (c & d);", "f = (b & c) ^ (b & d);"),
    "sha1_constant_sqrt3": ("{2.0, 3.0, 5.0, 10.0}", "{2.0, 2.0, 5.0, 10.0}"),
    "feature_digest_big_endian": ("h |= (uint64_t)dg[b] << (8 * b);", "h |= (uint64_t)dg[b] << (8 * (7 - b));"),
    "feature_seed_dropped": ("msg[4 + b] = (uint8_t)(seed >> (8 * b));", "msg[4 + b] = 0;"),
    "feature_md5_sha1_swapped": ("if (mode == 1) orc_md5(msg, 12, dg);", "if (mode == 2) orc_md5(msg, 12, dg);"),
    "hamming_counts_equal_bits": ("c += (int32_t)((x >> bit) & 1ULL);", "c += (int32_t)(((x >> bit) & 1ULL) ^ 1ULL);"),
    "pairs_include_self": ("for (int64_t j = i + 1; j < n; ++j) {\n            double c = orc_cos_dense",
                           "for (int64_t j = i; j < n; ++j) {\n            double c = orc_cos_dense"),
    "pairs_strict_threshold": ("double c = orc_cos_dense(S + i * k, S + j * k, k);\n            if (c >= tau)",
                               "double c = orc_cos_dense(S + i * k, S + j * k, k);\n            if (c > tau)"),
    "hamming_pairs_strict": ("if (h <= hmax)", "if (h < hmax)"),
    "error_stats_signed": ("sa += fabs(e);", "sa += e;"),
    "bf16_truncates": ("u += 0x7FFFu + ((u >> 16) & 1u);", "u += 0u;"),
    "bf16_ties_away": ("u += 0x7FFFu + ((u >> 16) & 1u);", "u += 0x8000u;"),
}


@pytest.fixture(scope="module")
def src():
    with open(obuild.SRC) as f:
        return f.read()


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_mutant_is_caught(tmp_path, src, name):
    old, new = MUTANTS[name]
    assert src.count(old) == 1, f"mutation site for {name} not unique/absent"
    path = tmp_path / f"mut_{name}.c"
    path.write_text(src.replace(old, new))
    lib = tmp_path / f"libmut_{name}.so"
    try:
        obuild.build(str(path), str(lib), force=True)
    except subprocess.CalledProcessError:
        pytest.fail(f"mutant {name} did not compile")
    failures = oracle_pins.run_all(Oracle(str(lib)))
    assert failures, f"no pin caught mutant {name}"


def test_unmutated_copy_passes(tmp_path, src):
    path = tmp_path / "copy.c"
    path.write_text(src)
    lib = tmp_path / "libcopy.so"
    obuild.build(str(path), str(lib), force=True)
    assert oracle_pins.run_all(Oracle(str(lib))) == []
