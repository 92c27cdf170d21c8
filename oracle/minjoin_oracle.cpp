// MinJoin oracle: plain, slow, obviously correct CPU restatement of the method
// of Zhang & Zhang, "MinJoin: Efficient Edit Similarity Joins via Local Hash
// Minima" (arXiv 1810.08833).
//
// TEST INFRASTRUCTURE ONLY.  Nothing on the product path may load this code:
// only the tests, the smoke check of the entry module and the CPU-baseline leg
// of the benchmark use it.  It shares no code, header, table or constant
// generator with the CUDA path.
//
// Each function follows the paper's steps in its order and notation, with
// 0-based positions in place of the paper's 1-based ones.  Readings of passages
// that are silent, ambiguous or garbled are stated where they are applied.
//
// Parity status: every function here is pinned by the CPU tests (worked
// example of Sec. 2.1, Tables 2-4; brute-force edit distance by breadth-first
// search; Lemma 1's anchor count; the set definition of the candidate pairs).

#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <string>
#include <unordered_map>
#include <utility>
#include <vector>

namespace {

// MurmurHash3 32-bit finaliser (A. Appleby, public domain): a bijection of
// 32-bit words with full avalanche.  Used as the random function Pi.
uint32_t fmix32(uint32_t h) {
    h ^= h >> 16;
    h *= 0x85ebca6bu;
    h ^= h >> 13;
    h *= 0xc2b2ae35u;
    h ^= h >> 16;
    return h;
}

// MurmurHash3 64-bit finaliser (same source), for q-grams wider than 32 bits.
uint64_t fmix64(uint64_t k) {
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}

int64_t floor_div(int64_t a, int64_t b) {  // b > 0
    int64_t q = a / b;
    if ((a % b != 0) && (a < 0)) q -= 1;
    return q;
}

int64_t iabs(int64_t x) { return x < 0 ? -x : x; }

}  // namespace

extern "C" {

// Sec. 2.2 (analysis assumptions): q = 3 log_|Sigma|(N/T).  Reading: rounded
// up, i.e. the smallest integer q >= 1 with |Sigma|^q >= (N/T)^3, decided
// exactly in integers as |Sigma|^q * T^3 >= N^3.  A one-symbol alphabet gives
// q = 1 (all q-grams are equal for every q).
uint32_t mjo_q_rule(uint64_t N, uint32_t T, uint32_t sigma) {
    if (sigma <= 1 || T == 0) return 1;
    unsigned __int128 t3 = (unsigned __int128)T * T * T;
    unsigned __int128 n3 = (unsigned __int128)N * N * N;
    unsigned __int128 p = 1;
    uint32_t q = 0;
    while (p * t3 < n3) {
        p *= sigma;
        q += 1;
    }
    return q < 1 ? 1 : q;
}

// Alg. 2, neighbourhood radius: r = floor((|s| - q + 1 - T) / (2T + 2)).  Reading: the
// division floors on signed integers, and r is raised to at least r_min
// (r_min = 0 keeps the literal rule wherever it is non-negative).
int64_t mjo_radius(int64_t slen, int64_t q, int64_t T, int64_t r_min) {
    int64_t r = floor_div(slen - q + 1 - T, 2 * T + 2);
    return r < r_min ? r_min : r;
}

// Alg. 2, q-gram values: h[i] = Pi(s[i .. i+q-1]) for every q-gram start i in
// [0, |s| - q].  Pi (Table 1: a random function Sigma^q -> (0,1)) is realised
// as: the q symbols, each replaced by its rank code of `bits` bits, packed
// first-symbol-most-significant into one integer `code`; then
//   Pi = fmix32(code ^ seed32)        when q*bits <= 32,
//   Pi = fmix64(code ^ seed)          otherwise,
// with seed32 = low32(seed) ^ high32(seed).  Both are bijections of the packed
// code, so two q-grams get equal values exactly when they are equal.  Values
// are compared as unsigned integers, the same order as a value in (0,1) with
// that many bits of precision.  If `table` is given, Pi(code) = table[code]
// instead (the explicit hash table of the worked example, Table 2).
void mjo_hash_qgrams(const uint8_t* s, int64_t slen, int32_t q, const uint8_t* rank,
                     int32_t bits, uint64_t seed, const uint64_t* table, uint64_t* h) {
    int64_t m = slen - q + 1;
    uint32_t seed32 = (uint32_t)seed ^ (uint32_t)(seed >> 32);
    for (int64_t i = 0; i < m; ++i) {
        uint64_t code = 0;
        for (int32_t t = 0; t < q; ++t) code = (code << bits) | (uint64_t)rank[s[i + t]];
        if (table) {
            h[i] = table[code];
        } else if ((int64_t)q * bits <= 32) {
            h[i] = fmix32((uint32_t)code ^ seed32);
        } else {
            h[i] = fmix64(code ^ seed);
        }
    }
}

// Alg. 2 (Find-Anchor), 0-based.  A starts as {0}; every i in
// [r, m-1-r] (m = |s| - q + 1 q-grams) whose value is strictly smaller than
// every other value within distance r is added; finally |s| is added.
// Reading of the closing anchor: the paper's 1-based "|s|" is taken as the
// exclusive end of the string (the worked example's last partitions run to the
// final symbol, Table 4), which is |s| in 0-based terms.  A is a set: the
// output is sorted and free of repeats.  Returns the number of anchors.
int64_t mjo_find_anchors(const uint64_t* h, int64_t m, int64_t slen, int64_t r, int64_t* anchors) {
    std::vector<int64_t> A;
    A.push_back(0);
    for (int64_t i = r; i <= m - 1 - r; ++i) {
        bool label = true;
        for (int64_t j = i - r; j <= i + r; ++j) {
            if (j == i) continue;
            if (h[i] >= h[j]) {
                label = false;
                break;
            }
        }
        if (label) A.push_back(i);
    }
    A.push_back(slen);
    std::sort(A.begin(), A.end());
    A.erase(std::unique(A.begin(), A.end()), A.end());
    for (size_t k = 0; k < A.size(); ++k) anchors[k] = A[k];
    return (int64_t)A.size();
}

// Alg. 1 (Partition-String) applied to strings [lo, hi) of a concatenated set.
// Reading of Alg. 1's partition pair: the pair emitted for anchor index i is
// (a_i, a_{i+1} - a_i) (the printed a_p is a typo).  Writes (sid, pos, len)
// triples in string order; returns their number, or -1 if `cap` is too small.
// `n_anchor` (optional) receives every string's anchor count.
int64_t mjo_partition_range(const uint8_t* bytes, const int64_t* offsets, int64_t lo, int64_t hi,
                            int32_t q, int64_t T, int64_t r_min, const uint8_t* rank, int32_t bits,
                            uint64_t seed, const uint64_t* table, int64_t* out_sid, int64_t* out_pos,
                            int64_t* out_len, int64_t cap, int64_t* n_anchor) {
    int64_t cnt = 0;
    std::vector<uint64_t> h;
    std::vector<int64_t> A;
    for (int64_t s = lo; s < hi; ++s) {
        const uint8_t* str = bytes + offsets[s];
        int64_t slen = offsets[s + 1] - offsets[s];
        int64_t m = slen - q + 1;
        int64_t r = mjo_radius(slen, q, T, r_min);
        h.assign(m > 0 ? (size_t)m : 0, 0);
        if (m > 0) mjo_hash_qgrams(str, slen, q, rank, bits, seed, table, h.data());
        A.assign((size_t)(m > 0 ? m : 0) + 2, 0);
        int64_t p = mjo_find_anchors(h.data(), m > 0 ? m : 0, slen, r, A.data());
        if (n_anchor) n_anchor[s - lo] = p;
        for (int64_t i = 0; i + 1 < p; ++i) {
            if (cnt >= cap) return -1;
            out_sid[cnt] = s;
            out_pos[cnt] = A[i];
            out_len[cnt] = A[i + 1] - A[i];
            ++cnt;
        }
    }
    return cnt;
}

// Alg. 3, the hash join: sort the strings by (length, alphabetical order), then
// for every string in that order and every partition (pos, len) of it, probe
// the bucket of the partition's substring in table D: an entry (j, pos_j,
// len_j) whose string length differs by more than K is evicted; otherwise
// the pair is a candidate if the position filter holds.  Then (i, pos, len)
// is stored in the bucket.  Duplicates are removed at the end.
// Readings: the bucket of f is the exact substring (no hash collisions can
// merge different substrings), and a string never pairs with itself (the
// output set of the algorithm requires i != j), which arises when one string
// has two equal partitions.  Partitions are given (sid, pos, len) sorted by
// sid, as written by mjo_partition_range.  Returns the number of distinct
// pairs (i < j) and sets *out to a malloc'd array of 2 * count int64 values
// (free with mjo_free).
int64_t mjo_candidates(const uint8_t* bytes, const int64_t* offsets, int64_t n, int64_t K,
                       const int64_t* part_sid, const int64_t* part_pos, const int64_t* part_len,
                       int64_t nparts, int64_t** out) {
    struct Entry {
        int64_t j, pos, len;
    };
    std::vector<int64_t> first(n + 1, 0);
    for (int64_t t = 0; t < nparts; ++t) first[part_sid[t] + 1] += 1;
    for (int64_t s = 0; s < n; ++s) first[s + 1] += first[s];

    std::vector<int64_t> order(n);
    for (int64_t s = 0; s < n; ++s) order[s] = s;
    auto len_of = [&](int64_t s) { return offsets[s + 1] - offsets[s]; };
    std::sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
        int64_t la = len_of(a), lb = len_of(b);
        if (la != lb) return la < lb;
        int c = std::memcmp(bytes + offsets[a], bytes + offsets[b], (size_t)la);
        if (c != 0) return c < 0;
        return a < b;
    });

    std::unordered_map<std::string, std::vector<Entry>> D;
    std::vector<std::pair<int64_t, int64_t>> C;
    for (int64_t i : order) {
        int64_t slen_i = len_of(i);
        for (int64_t t = first[i]; t < first[i + 1]; ++t) {
            int64_t pos = part_pos[t], len = part_len[t];
            std::string key((const char*)(bytes + offsets[i] + pos), (size_t)len);
            std::vector<Entry>& bucket = D[key];
            std::vector<Entry> kept;
            kept.reserve(bucket.size() + 1);
            for (const Entry& e : bucket) {
                int64_t slen_j = len_of(e.j);
                if (iabs(slen_i - slen_j) <= K) {
                    if (iabs(pos - e.pos) + iabs((slen_i - pos) - (slen_j - e.pos)) <= K && e.j != i)
                        C.emplace_back(std::min(i, e.j), std::max(i, e.j));
                    kept.push_back(e);
                }
                // else: evicted from D (length filter)
            }
            kept.push_back(Entry{i, pos, len});
            bucket.swap(kept);
        }
    }
    std::sort(C.begin(), C.end());
    C.erase(std::unique(C.begin(), C.end()), C.end());
    int64_t* buf = (int64_t*)std::malloc(sizeof(int64_t) * 2 * (C.size() ? C.size() : 1));
    for (size_t k = 0; k < C.size(); ++k) {
        buf[2 * k] = C[k].first;
        buf[2 * k + 1] = C[k].second;
    }
    *out = buf;
    return (int64_t)C.size();
}

void mjo_free(void* p) { std::free(p); }

// Sec. 1 (problem statement): ED is the minimum number of insertions,
// deletions and substitutions turning one string into the other.  Textbook
// dynamic program D[i][j] = min(D[i-1][j] + 1, D[i][j-1] + 1,
// D[i-1][j-1] + [a_i != b_j]) with D[i][0] = i, D[0][j] = j.
int64_t mjo_ed_full(const uint8_t* a, int64_t m, const uint8_t* b, int64_t n) {
    std::vector<int64_t> prev(n + 1), cur(n + 1);
    for (int64_t j = 0; j <= n; ++j) prev[j] = j;
    for (int64_t i = 1; i <= m; ++i) {
        cur[0] = i;
        for (int64_t j = 1; j <= n; ++j) {
            int64_t v = prev[j - 1] + (a[i - 1] != b[j - 1] ? 1 : 0);
            v = std::min(v, prev[j] + 1);
            v = std::min(v, cur[j - 1] + 1);
            cur[j] = v;
        }
        std::swap(prev, cur);
    }
    return prev[n];
}

// Sec. 3 (verification, Ukkonen's banded dynamic program): the same recurrence
// restricted to cells with |i - j| <= k, every cell outside the band being
// infinite.  Reading: the returned value is ED when ED <= k and k + 1
// otherwise (a pair whose lengths differ by more than k is k + 1 at once).
int64_t mjo_ed_band(const uint8_t* a, int64_t m, const uint8_t* b, int64_t n, int64_t k) {
    if (iabs(m - n) > k) return k + 1;
    const int64_t INF = k + 1;
    std::vector<int64_t> prev(n + 1, INF), cur(n + 1, INF);
    for (int64_t j = 0; j <= std::min(n, k); ++j) prev[j] = j;
    for (int64_t i = 1; i <= m; ++i) {
        int64_t jlo = std::max<int64_t>(0, i - k), jhi = std::min(n, i + k);
        // only band cells are read: (i-1, j-1) always lies in the band with
        // (i, j); the other two neighbours are tested explicitly
        for (int64_t j = jlo; j <= jhi; ++j) {
            int64_t v = INF;
            if (j == 0) {
                v = i;
            } else {
                v = prev[j - 1] + (a[i - 1] != b[j - 1] ? 1 : 0);  // (i-1, j-1) is in band
                if (iabs((i - 1) - j) <= k) v = std::min(v, prev[j] + 1);
                if (j - 1 >= jlo) v = std::min(v, cur[j - 1] + 1);
            }
            cur[j] = std::min(v, INF);
        }
        std::swap(prev, cur);
    }
    return std::min(prev[n], INF);
}

// mjo_ed_band with the cut-off of Ukkonen's method (Sec. 3 names Ukkonen's
// algorithm for the verification): the dynamic program stops as soon as every
// band cell of a row exceeds k and returns k + 1.  That is exact: each cell of
// row i is reached from a cell of row i - 1 (diagonal or vertical step) or
// from a cell of row i to its left, and no step lowers the cost, so the
// smallest band value of a row never falls below that of the row above, and
// the final cell (m, n) can no longer be within k.  Otherwise the same
// recurrence, boundary and band as mjo_ed_band.
int64_t mjo_ed_band_cutoff(const uint8_t* a, int64_t m, const uint8_t* b, int64_t n, int64_t k) {
    if (iabs(m - n) > k) return k + 1;
    const int64_t INF = k + 1;
    std::vector<int64_t> prev(n + 1, INF), cur(n + 1, INF);
    for (int64_t j = 0; j <= std::min(n, k); ++j) prev[j] = j;
    for (int64_t i = 1; i <= m; ++i) {
        int64_t jlo = std::max<int64_t>(0, i - k), jhi = std::min(n, i + k);
        int64_t row_min = INF;
        for (int64_t j = jlo; j <= jhi; ++j) {
            int64_t v = INF;
            if (j == 0) {
                v = i;
            } else {
                v = prev[j - 1] + (a[i - 1] != b[j - 1] ? 1 : 0);
                if (iabs((i - 1) - j) <= k) v = std::min(v, prev[j] + 1);
                if (j - 1 >= jlo) v = std::min(v, cur[j - 1] + 1);
            }
            cur[j] = std::min(v, INF);
            row_min = std::min(row_min, cur[j]);
        }
        if (row_min > k) return k + 1;
        std::swap(prev, cur);
    }
    return std::min(prev[n], INF);
}

// mjo_ed_band over pairs [lo, hi) of a pair list (pairs[2t], pairs[2t+1]).
void mjo_ed_band_pairs(const uint8_t* bytes, const int64_t* offsets, const int64_t* pairs,
                       int64_t lo, int64_t hi, int64_t k, int64_t* out) {
    for (int64_t t = lo; t < hi; ++t) {
        int64_t x = pairs[2 * t], y = pairs[2 * t + 1];
        out[t] = mjo_ed_band(bytes + offsets[x], offsets[x + 1] - offsets[x], bytes + offsets[y],
                             offsets[y + 1] - offsets[y], k);
    }
}

// mjo_ed_band_cutoff over pairs [lo, hi) of a pair list, as mjo_ed_band_pairs.
void mjo_ed_band_cutoff_pairs(const uint8_t* bytes, const int64_t* offsets, const int64_t* pairs,
                              int64_t lo, int64_t hi, int64_t k, int64_t* out) {
    for (int64_t t = lo; t < hi; ++t) {
        int64_t x = pairs[2 * t], y = pairs[2 * t + 1];
        out[t] = mjo_ed_band_cutoff(bytes + offsets[x], offsets[x + 1] - offsets[x], bytes + offsets[y],
                                    offsets[y + 1] - offsets[y], k);
    }
}

}  // extern "C"
