"""The FP64 oracle against values and invariants that do not come from the oracle.

Parity status of the oracle's functions (every function is pinned):
  orc_splitmix64 / orc_term_hash  published SplitMix64 outputs
  orc_md5 / orc_sha1               RFC 1321 test suite, FIPS 180 examples; hashlib, lengths 0-130
  orc_feature_hash                 hashlib on the 12-byte term/seed message, all three modes
  orc_char3grams                   hand-numbered 3-grams; regular-expression brute force, run-length counts
  orc_idf                          hand-evaluated closed forms
  orc_term_counts, orc_df          hand example; brute force
  orc_select_refs                  hand-ranked example for all three modes; brute force
  orc_ref_norms, orc_signatures    hand closed form; one-hot reference documents;
                                   singleton-partition limit equals exact cosine; brute force
  orc_cos_dense, orc_cosine_pair   symmetry, cos(x,x)=1, scaled/disjoint docs; brute force
  orc_simhash, orc_hamming         one/two/three-term closed forms (each hash mode); textbook popcount
  orc_*_pairs                      emission rules by hand; brute-force pair sets
  orc_error_stats                  hand example
"""
import pytest

from oracle.oracle import Oracle
from tests import oracle_pins


@pytest.fixture(scope="module")
def orc():
    return Oracle()


@pytest.mark.parametrize("pin", oracle_pins.ALL_PINS, ids=lambda f: f.__name__)
def test_pin(orc, pin):
    pin(orc)
