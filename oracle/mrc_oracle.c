/*
 * mrc_oracle.c -- FP64 CPU oracle for Multi-reference Cosine (arXiv 1810.03099).
 *
 * TEST INFRASTRUCTURE ONLY. The tests, the smoke check and the benchmark's CPU
 * baseline call this library; the product path (the CUDA library) never does.
 * It shares no code, header, table or constant generator with the CUDA path.
 *
 * Every function is the plain definition written out with loops in double
 * precision; there is no blocking, fusion or reordering. Where the paper is
 * silent or ambiguous, the reading taken is stated at the function.
 *
 * Data layout: a corpus is a token CSR (offsets[n+1] int64, tokens[T] int32,
 * a token id stands for one character 3-gram of Section III). A count CSR
 * (row_ptr[n+1], terms[], counts[]) holds each document's distinct terms in
 * ascending id order with their occurrence counts.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_MODE_ALL 0
#define ORC_MODE_REGION 1
#define ORC_MODE_DF1 2

static int cmp_i32(const void* a, const void* b) {
    int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
    return (x > y) - (x < y);
}

/*
 * Character 3-grams of raw text (Section III: a document is the vector of its
 * N-gram counts, N = 3; an N-gram is a sequence of N letters of the alphabet).
 * Reading taken: the alphabet is the 26 ASCII letters with case folded
 * (A-Z equal a-z), so there are 26^3 = 17,576 possible 3-grams; every other
 * byte separates, and a 3-gram is any 3 consecutive letters of a document
 * (a letter run of length m gives m - 2 of them). The 3-gram (x, y, z), each
 * letter numbered 0..25, has id 676 x + 26 y + z. Document d is the bytes
 * [text_offsets[d], text_offsets[d+1]); its 3-gram ids are written in text
 * order. grams needs room for text_offsets[n] entries. Returns the total.
 */
static int orc_letter(uint8_t c) {
    if (c >= 'a' && c <= 'z') return c - 'a';
    if (c >= 'A' && c <= 'Z') return c - 'A';
    return -1;
}

int64_t orc_char3grams(int64_t n, const int64_t* text_offsets, const uint8_t* text, int64_t* gram_offsets,
                       int32_t* grams) {
    int64_t out = 0;
    gram_offsets[0] = 0;
    for (int64_t d = 0; d < n; ++d) {
        for (int64_t p = text_offsets[d]; p + 2 < text_offsets[d + 1]; ++p) {
            int x = orc_letter(text[p]), y = orc_letter(text[p + 1]), z = orc_letter(text[p + 2]);
            if (x >= 0 && y >= 0 && z >= 0) grams[out++] = 676 * x + 26 * y + z;
        }
        gram_offsets[d + 1] = out;
    }
    return out;
}

/*
 * Term counts of each document (Section III: a document becomes the vector of
 * its N-gram counts). Output rows are sorted by term id. Capacity of
 * terms/counts must be >= offsets[n]. Returns the number of entries written.
 */
int64_t orc_term_counts(int64_t n, const int64_t* offsets, const int32_t* tokens,
                        int64_t* row_ptr, int32_t* terms, int32_t* counts) {
    int64_t out = 0;
    row_ptr[0] = 0;
    for (int64_t d = 0; d < n; ++d) {
        int64_t len = offsets[d + 1] - offsets[d];
        int32_t* tmp = (int32_t*)malloc(sizeof(int32_t) * (size_t)(len > 0 ? len : 1));
        memcpy(tmp, tokens + offsets[d], sizeof(int32_t) * (size_t)len);
        qsort(tmp, (size_t)len, sizeof(int32_t), cmp_i32);
        for (int64_t x = 0; x < len;) {
            int64_t y = x;
            while (y < len && tmp[y] == tmp[x]) ++y;
            terms[out] = tmp[x];
            counts[out] = (int32_t)(y - x);
            ++out;
            x = y;
        }
        free(tmp);
        row_ptr[d + 1] = out;
    }
    return out;
}

/* Document frequency: number of documents containing each term. */
void orc_df(int64_t n, const int64_t* row_ptr, const int32_t* terms, int32_t vocab, int64_t* df) {
    for (int32_t t = 0; t < vocab; ++t) df[t] = 0;
    for (int64_t d = 0; d < n; ++d)
        for (int64_t e = row_ptr[d]; e < row_ptr[d + 1]; ++e) df[terms[e]] += 1;
}

/*
 * Inverse document frequency. The paper defines no weighting (its future work,
 * Section VI, names weighted vector space models). Reading taken: the smoothed
 * form idf(t) = ln((1 + N) / (1 + df(t))) + 1, which is >= 1 for every term.
 */
void orc_idf(int64_t n_docs, int32_t vocab, const int64_t* df, double* idf) {
    for (int32_t t = 0; t < vocab; ++t)
        idf[t] = log((1.0 + (double)n_docs) / (1.0 + (double)df[t])) + 1.0;
}

/*
 * Reduced-precision storage of the per-term weights (the precision form): a
 * value is rounded to FP32, then to bfloat16 (8 significant bits, round to
 * nearest, ties to even). out[t] = that value, for every term.
 */
double orc_round_bf16(double x) {
  float f = (float)x;
  uint32_t u;
  memcpy(&u, &f, sizeof(u));
  u += 0x7FFFu + ((u >> 16) & 1u);
  u &= 0xFFFF0000u;
  memcpy(&f, &u, sizeof(f));
  return (double)f;
}

void orc_idf_bf16(int32_t vocab, const double* idf, double* out) {
  for (int32_t t = 0; t < vocab; ++t) out[t] = orc_round_bf16(idf[t]);
}

/* w(d,t) = c(d,t) * idf(t); with idf == NULL, w = c (the paper's plain counts). */
void orc_weights(int64_t nnz, const int32_t* terms, const int32_t* counts, const double* idf, double* w) {
    for (int64_t e = 0; e < nnz; ++e) w[e] = (double)counts[e] * (idf ? idf[terms[e]] : 1.0);
}

/*
 * Default start of a frequency region (Section IV): the first rank whose df is
 * at most N/100, which skips the terms present in almost every document (the
 * paper's "the"/"and" remark). Ranks order terms by df descending, then id.
 */
typedef struct { int64_t df; int32_t t; } orc_rank_entry;

static int cmp_rank(const void* a, const void* b) {
    const orc_rank_entry* x = (const orc_rank_entry*)a;
    const orc_rank_entry* y = (const orc_rank_entry*)b;
    if (x->df != y->df) return (x->df < y->df) - (x->df > y->df); /* df descending */
    return (x->t > y->t) - (x->t < y->t);                          /* id ascending */
}

/*
 * Reference selection and partitioning (Section IV).
 *   ALL    : every term of non-zero df, in rank order (the all-3-gram reference
 *            with zero-frequency 3-grams removed).
 *   REGION : ranks [start, start + L) of the frequency-sorted list; start < 0
 *            takes the default above.
 *   DF1    : the first L terms (id order) that occur in exactly one document.
 * The L selected terms are split into k contiguous partitions of (near) equal
 * length: partition p holds selection positions [floor(pL/k), floor((p+1)L/k)).
 * Reading taken: a partition is the set of its terms (the paper concatenates
 * 3-grams into one string; splitting that string would create 3-grams that
 * straddle the cut, which are not counted here).
 * part[t] receives the partition of term t, or -1. Returns the number of
 * selected terms L_used, or -1 on invalid arguments.
 */
int64_t orc_select_refs(int32_t vocab, int64_t n_docs, const int64_t* df, int32_t mode, int64_t L,
                        int64_t start, int32_t k, int32_t* part) {
    if (k <= 0 || vocab <= 0) return -1;
    for (int32_t t = 0; t < vocab; ++t) part[t] = -1;
    int32_t* sel = (int32_t*)malloc(sizeof(int32_t) * (size_t)vocab);
    int64_t n_sel = 0;
    if (mode == ORC_MODE_DF1) {
        for (int32_t t = 0; t < vocab && n_sel < L; ++t)
            if (df[t] == 1) sel[n_sel++] = t;
    } else {
        orc_rank_entry* r = (orc_rank_entry*)malloc(sizeof(orc_rank_entry) * (size_t)vocab);
        int64_t nr = 0;
        for (int32_t t = 0; t < vocab; ++t)
            if (df[t] > 0) { r[nr].df = df[t]; r[nr].t = t; ++nr; }
        qsort(r, (size_t)nr, sizeof(orc_rank_entry), cmp_rank);
        if (mode == ORC_MODE_ALL) {
            for (int64_t q = 0; q < nr; ++q) sel[n_sel++] = r[q].t;
        } else if (mode == ORC_MODE_REGION) {
            if (start < 0) {
                start = nr;
                for (int64_t q = 0; q < nr; ++q)
                    if ((double)r[q].df <= (double)n_docs / 100.0) { start = q; break; }
            }
            for (int64_t q = start; q < nr && q < start + L; ++q) sel[n_sel++] = r[q].t;
        } else {
            free(r); free(sel);
            return -1;
        }
        free(r);
    }
    for (int32_t p = 0; p < k; ++p) {
        int64_t lo = ((int64_t)p * n_sel) / k;
        int64_t hi = ((int64_t)(p + 1) * n_sel) / k;
        for (int64_t q = lo; q < hi; ++q) part[sel[q]] = p;
    }
    free(sel);
    return n_sel;
}

/*
 * |R_p|: norm of each reference partition's vector. Each reference term occurs
 * once in its partition, so its weight is 1 * idf(t) (counts: 1), i.e. a
 * reference is weighted exactly like a document.
 */
void orc_ref_norms(int32_t vocab, const int32_t* part, int32_t k, const double* idf, double* rnorm) {
    for (int32_t p = 0; p < k; ++p) rnorm[p] = 0.0;
    for (int32_t t = 0; t < vocab; ++t)
        if (part[t] >= 0) {
            double r = idf ? idf[t] : 1.0;
            rnorm[part[t]] += r * r;
        }
    for (int32_t p = 0; p < k; ++p) rnorm[p] = sqrt(rnorm[p]);
}

/*
 * MRC signature (Section IV): entry p is the cosine (Eq. 1) between the
 * document's vector and reference partition p,
 *   s_p(d) = sum_{t in R_p} w(d,t) r_t / (|d| |R_p|),
 * |d| taken over all of d's terms. A zero norm on either side gives 0.
 */
void orc_signatures(int64_t n, const int64_t* row_ptr, const int32_t* terms, const double* w,
                    const int32_t* part, const double* idf, const double* rnorm, int32_t k, double* S) {
    for (int64_t d = 0; d < n; ++d) {
        double* s = S + d * k;
        for (int32_t p = 0; p < k; ++p) s[p] = 0.0;
        double nrm = 0.0;
        for (int64_t e = row_ptr[d]; e < row_ptr[d + 1]; ++e) nrm += w[e] * w[e];
        nrm = sqrt(nrm);
        for (int64_t e = row_ptr[d]; e < row_ptr[d + 1]; ++e) {
            int32_t p = part[terms[e]];
            if (p >= 0) s[p] += w[e] * (idf ? idf[terms[e]] : 1.0);
        }
        for (int32_t p = 0; p < k; ++p)
            s[p] = (nrm > 0.0 && rnorm[p] > 0.0) ? s[p] / (nrm * rnorm[p]) : 0.0;
    }
}

/*
 * Signature similarity, the "multi reference cosine" of Eq. 2. The paper never
 * writes it out; reading taken: the cosine (Eq. 1) of the two signature
 * vectors. A zero signature has similarity 0 with everything.
 */
double orc_cos_dense(const double* a, const double* b, int32_t k) {
    double ab = 0.0, aa = 0.0, bb = 0.0;
    for (int32_t p = 0; p < k; ++p) {
        ab += a[p] * b[p];
        aa += a[p] * a[p];
        bb += b[p] * b[p];
    }
    if (aa <= 0.0 || bb <= 0.0) return 0.0;
    return ab / (sqrt(aa) * sqrt(bb));
}

/* Exact cosine (Eq. 1) of two count-CSR rows: merge of the sorted term lists. */
double orc_cosine_rows(const int32_t* ti, const double* wi, int64_t ni,
                       const int32_t* tj, const double* wj, int64_t nj) {
    double ab = 0.0, aa = 0.0, bb = 0.0;
    for (int64_t x = 0; x < ni; ++x) aa += wi[x] * wi[x];
    for (int64_t y = 0; y < nj; ++y) bb += wj[y] * wj[y];
    int64_t x = 0, y = 0;
    while (x < ni && y < nj) {
        if (ti[x] == tj[y]) { ab += wi[x] * wj[y]; ++x; ++y; }
        else if (ti[x] < tj[y]) ++x;
        else ++y;
    }
    if (aa <= 0.0 || bb <= 0.0) return 0.0;
    return ab / (sqrt(aa) * sqrt(bb));
}

double orc_cosine_pair(const int64_t* row_ptr, const int32_t* terms, const double* w, int64_t i, int64_t j) {
    return orc_cosine_rows(terms + row_ptr[i], w + row_ptr[i], row_ptr[i + 1] - row_ptr[i],
                           terms + row_ptr[j], w + row_ptr[j], row_ptr[j + 1] - row_ptr[j]);
}

/* Pair emission: every i < j whose similarity is >= tau (inclusive). The total
 * is returned; at most cap pairs are stored, in (i, j) lexicographic order. */
int64_t orc_sig_pairs(const double* S, int64_t n, int32_t k, double tau,
                      int32_t* pi, int32_t* pj, double* ps, int64_t cap) {
    int64_t cnt = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) {
            double c = orc_cos_dense(S + i * k, S + j * k, k);
            if (c >= tau) {
                if (cnt < cap) { pi[cnt] = (int32_t)i; pj[cnt] = (int32_t)j; ps[cnt] = c; }
                ++cnt;
            }
        }
    return cnt;
}

/* Query x index signature match: every (q, x) with similarity >= tau. */
int64_t orc_sig_match(const double* Q, int64_t nq, const double* X, int64_t nx, int32_t k, double tau,
                      int32_t* pi, int32_t* pj, double* ps, int64_t cap) {
    int64_t cnt = 0;
    for (int64_t i = 0; i < nq; ++i)
        for (int64_t j = 0; j < nx; ++j) {
            double c = orc_cos_dense(Q + i * k, X + j * k, k);
            if (c >= tau) {
                if (cnt < cap) { pi[cnt] = (int32_t)i; pj[cnt] = (int32_t)j; ps[cnt] = c; }
                ++cnt;
            }
        }
    return cnt;
}

/* Exact-cosine pairs over a count CSR with weights w. */
int64_t orc_cosine_pairs(int64_t n, const int64_t* row_ptr, const int32_t* terms, const double* w,
                         double tau, int32_t* pi, int32_t* pj, double* ps, int64_t cap) {
    int64_t cnt = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j) {
            double c = orc_cosine_pair(row_ptr, terms, w, i, j);
            if (c >= tau) {
                if (cnt < cap) { pi[cnt] = (int32_t)i; pj[cnt] = (int32_t)j; ps[cnt] = c; }
                ++cnt;
            }
        }
    return cnt;
}

/*
 * 64-bit feature hash. The paper hashes words with MD5 or SHA1 (Section III);
 * those two are hash modes 1 and 2 below. Default reading (mode 0): the
 * SplitMix64 generator of Steele, Lea and Flood (2014),
 * one step from state (t XOR seed): add the golden-ratio increment
 * 0x9E3779B97F4A7C15, then the two xor-shift-multiply rounds with the
 * published multipliers and a final xor-shift.
 */
uint64_t orc_splitmix64(uint64_t state) {
    uint64_t z = state + 0x9E3779B97F4A7C15ULL;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

uint64_t orc_term_hash(int32_t t, uint64_t seed) { return orc_splitmix64((uint64_t)(uint32_t)t ^ seed); }

/*
 * MD5 (RFC 1321) of a byte message; digest[16] receives the four state words
 * as little-endian bytes. The message is padded with one 0x80 byte, zeros up
 * to 56 mod 64 bytes, then its length in bits as a little-endian 64-bit word,
 * and processed in 64-byte blocks of sixteen little-endian words. The additive
 * constant of step i (1..64) is floor(2^32 * |sin(i)|), computed here from
 * that definition.
 */
static uint32_t orc_rotl32(uint32_t x, int s) { return (x << s) | (x >> (32 - s)); }

static uint8_t orc_pad_byte_le(const uint8_t* msg, int64_t len, int64_t padded, int64_t pos) {
    if (pos < len) return msg[pos];
    if (pos == len) return 0x80;
    if (pos >= padded - 8) return (uint8_t)(((uint64_t)len * 8u) >> (8 * (pos - (padded - 8))));
    return 0;
}

void orc_md5(const uint8_t* msg, int64_t len, uint8_t* digest) {
    static const int shift[4][4] = {{7, 12, 17, 22}, {5, 9, 14, 20}, {4, 11, 16, 23}, {6, 10, 15, 21}};
    uint32_t T[64];
    for (int i = 0; i < 64; ++i) T[i] = (uint32_t)floor(4294967296.0 * fabs(sin((double)(i + 1))));
    uint32_t state[4] = {0x67452301u, 0xEFCDAB89u, 0x98BADCFEu, 0x10325476u};
    const int64_t padded = (len + 9 + 63) / 64 * 64;
    for (int64_t blk = 0; blk < padded; blk += 64) {
        uint32_t X[16];
        for (int w = 0; w < 16; ++w) {
            uint32_t v = 0;
            for (int b = 3; b >= 0; --b) v = (v << 8) | orc_pad_byte_le(msg, len, padded, blk + 4 * w + b);
            X[w] = v;
        }
        uint32_t a = state[0], b = state[1], c = state[2], d = state[3];
        for (int i = 0; i < 64; ++i) {
            const int round = i / 16;
            uint32_t f;
            int k;
            if (round == 0) {        /* F(X,Y,Z) = XY v not(X) Z */
                f = (b & c) | (~b & d);
                k = i;
            } else if (round == 1) { /* G(X,Y,Z) = XZ v Y not(Z) */
                f = (b & d) | (c & ~d);
                k = (1 + 5 * i) % 16;
            } else if (round == 2) { /* H(X,Y,Z) = X xor Y xor Z */
                f = b ^ c ^ d;
                k = (5 + 3 * i) % 16;
            } else {                 /* I(X,Y,Z) = Y xor (X v not(Z)) */
                f = c ^ (b | ~d);
                k = (7 * i) % 16;
            }
            /* a = b + ((a + f(b,c,d) + X[k] + T[i]) <<< s), then the roles of a, b, c, d rotate */
            const uint32_t nb = b + orc_rotl32(a + f + X[k] + T[i], shift[round][i % 4]);
            a = d;
            d = c;
            c = b;
            b = nb;
        }
        state[0] += a;
        state[1] += b;
        state[2] += c;
        state[3] += d;
    }
    for (int w = 0; w < 4; ++w)
        for (int b = 0; b < 4; ++b) digest[4 * w + b] = (uint8_t)(state[w] >> (8 * b));
}

/*
 * SHA-1 (FIPS 180-4, Section 6.1) of a byte message; digest[20] receives the
 * five state words as big-endian bytes. Padding as MD5's but with the bit
 * length and the message words big-endian. The round constants are
 * floor(2^30 * sqrt(n)) for n = 2, 3, 5, 10, computed here from that
 * definition.
 */
static uint8_t orc_pad_byte_be(const uint8_t* msg, int64_t len, int64_t padded, int64_t pos) {
    if (pos < len) return msg[pos];
    if (pos == len) return 0x80;
    if (pos >= padded - 8) return (uint8_t)(((uint64_t)len * 8u) >> (8 * (7 - (pos - (padded - 8)))));
    return 0;
}

void orc_sha1(const uint8_t* msg, int64_t len, uint8_t* digest) {
    static const double radicand[4] = {2.0, 3.0, 5.0, 10.0};
    uint32_t K[4];
    for (int q = 0; q < 4; ++q) K[q] = (uint32_t)floor(1073741824.0 * sqrt(radicand[q]));
    uint32_t H[5] = {0x67452301u, 0xEFCDAB89u, 0x98BADCFEu, 0x10325476u, 0xC3D2E1F0u};
    const int64_t padded = (len + 9 + 63) / 64 * 64;
    for (int64_t blk = 0; blk < padded; blk += 64) {
        uint32_t W[80];
        for (int t = 0; t < 16; ++t) {
            uint32_t v = 0;
            for (int b = 0; b < 4; ++b) v = (v << 8) | orc_pad_byte_be(msg, len, padded, blk + 4 * t + b);
            W[t] = v;
        }
        for (int t = 16; t < 80; ++t) W[t] = orc_rotl32(W[t - 3] ^ W[t - 8] ^ W[t - 14] ^ W[t - 16], 1);
        uint32_t a = H[0], b = H[1], c = H[2], d = H[3], e = H[4];
        for (int t = 0; t < 80; ++t) {
            uint32_t f;
            if (t < 20) f = (b & c) ^ (~b & d);             /* Ch */
            else if (t < 40) f = b ^ c ^ d;                 /* Parity */
            else if (t < 60) f = (b & c) ^ (b & d) ^ (c & d); /* Maj */
            else f = b ^ c ^ d;                             /* Parity */
            const uint32_t T = orc_rotl32(a, 5) + f + e + K[t / 20] + W[t];
            e = d;
            d = c;
            c = orc_rotl32(b, 30);
            b = a;
            a = T;
        }
        H[0] += a;
        H[1] += b;
        H[2] += c;
        H[3] += d;
        H[4] += e;
    }
    for (int w = 0; w < 5; ++w)
        for (int b = 0; b < 4; ++b) digest[4 * w + b] = (uint8_t)(H[w] >> (24 - 8 * b));
}

/*
 * The 64-bit feature hash of term t under each hash mode. Mode 0 is the
 * SplitMix64 step above. Modes 1 (MD5) and 2 (SHA-1) are the paper's hashes
 * (Section III), applied to a 12-byte message: t as a 32-bit little-endian
 * word, then the seed as a 64-bit little-endian word; the feature is the
 * first 8 digest bytes read as a little-endian word (bit b of the feature is
 * bit b % 8 of digest byte b / 8).
 */
uint64_t orc_feature_hash(int32_t t, uint64_t seed, int32_t mode) {
    if (mode == 0) return orc_term_hash(t, seed);
    uint8_t msg[12], dg[20];
    for (int b = 0; b < 4; ++b) msg[b] = (uint8_t)((uint32_t)t >> (8 * b));
    for (int b = 0; b < 8; ++b) msg[4 + b] = (uint8_t)(seed >> (8 * b));
    if (mode == 1) orc_md5(msg, 12, dg);
    else orc_sha1(msg, 12, dg);
    uint64_t h = 0;
    for (int b = 0; b < 8; ++b) h |= (uint64_t)dg[b] << (8 * b);
    return h;
}

/*
 * Simhash (Section III): every token occurrence is hashed to 64 bits (feature
 * hash mode `mode`); bit column b adds +1 where the bit is 1 and -1 where it
 * is 0; result bit b is 1 iff the column sum is strictly greater than 0 (a tie
 * gives 0). Bit b of the result is (F >> b) & 1.
 */
void orc_simhash(int64_t n, const int64_t* offsets, const int32_t* tokens, uint64_t seed, int32_t mode, uint64_t* F) {
    for (int64_t d = 0; d < n; ++d) {
        int64_t col[64];
        for (int b = 0; b < 64; ++b) col[b] = 0;
        for (int64_t x = offsets[d]; x < offsets[d + 1]; ++x) {
            uint64_t h = orc_feature_hash(tokens[x], seed, mode);
            for (int b = 0; b < 64; ++b) col[b] += ((h >> b) & 1ULL) ? 1 : -1;
        }
        uint64_t f = 0;
        for (int b = 0; b < 64; ++b)
            if (col[b] > 0) f |= (1ULL << b);
        F[d] = f;
    }
}

/* Hamming distance: the number of bit positions in which the two words differ. */
int32_t orc_hamming(uint64_t a, uint64_t b) {
    uint64_t x = a ^ b;
    int32_t c = 0;
    for (int bit = 0; bit < 64; ++bit) c += (int32_t)((x >> bit) & 1ULL);
    return c;
}

/* Simhash pairs: all i < j (b == NULL) or all (i in a, j in b) with H <= hmax. */
int64_t orc_hamming_pairs(const uint64_t* a, int64_t na, const uint64_t* b, int64_t nb, int32_t hmax,
                          int32_t* pi, int32_t* pj, int32_t* ph, int64_t cap) {
    int64_t cnt = 0;
    for (int64_t i = 0; i < na; ++i) {
        int64_t j0 = b ? 0 : i + 1;
        const uint64_t* other = b ? b : a;
        int64_t no = b ? nb : na;
        for (int64_t j = j0; j < no; ++j) {
            int32_t h = orc_hamming(a[i], other[j]);
            if (h <= hmax) {
                if (cnt < cap) { pi[cnt] = (int32_t)i; pj[cnt] = (int32_t)j; ph[cnt] = h; }
                ++cnt;
            }
        }
    }
    return cnt;
}

/*
 * Error of a similarity against the exact cosine over all pairs i < j (Eq. 2
 * and Eq. 3). The printed Eq. 2 has no absolute value and divides by the
 * number of documents; reading taken: MAE = mean over the n(n-1)/2 pairs of
 * |approx - exact|. Eq. 3's "mean distance" is undefined; the spread reported
 * is the variance of the signed error e = approx - exact around its mean.
 * out[0] = MAE, out[1] = mean signed error, out[2] = Var(e), out[3] = E[e^2].
 */
void orc_error_stats(const double* approx, const double* exact, int64_t m, double* out) {
    double sa = 0.0, s = 0.0, s2 = 0.0;
    for (int64_t x = 0; x < m; ++x) {
        double e = approx[x] - exact[x];
        sa += fabs(e);
        s += e;
        s2 += e * e;
    }
    double mean = m ? s / (double)m : 0.0;
    double var = 0.0;
    for (int64_t x = 0; x < m; ++x) {
        double e = approx[x] - exact[x] - mean;
        var += e * e;
    }
    out[0] = m ? sa / (double)m : 0.0;
    out[1] = mean;
    out[2] = m ? var / (double)m : 0.0;
    out[3] = m ? s2 / (double)m : 0.0;
}
