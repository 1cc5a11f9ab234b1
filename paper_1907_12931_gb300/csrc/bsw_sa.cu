// bsw_sa.cu - suffix array construction for the suffix-array lookup (host).
//
// Section IV-D: with the suffix array S of the reference kept uncompressed,
// a lookup is j = S[i] (Eq. 1).  This file builds S once per reference (an
// index step, not the lookup path): the suffix array of text + "$", where $
// is smaller than every base, so S[0] = n.  The construction is induced
// sorting (SA-IS: Nong, Zhang and Chan, "Two efficient algorithms for linear
// time suffix array construction", IEEE Trans. Computers 2011): classify
// every suffix as S- or L-type, sort the leftmost-S (LMS) suffixes by sorting
// their substrings with two induction passes, name them, recurse when names
// repeat, and induce the order of all suffixes from the sorted LMS suffixes.
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "bsw.h"

namespace {

using idx_t = int32_t;

// Start (head) or end (tail) of each symbol's bucket in SA.
void bucket_bounds(const idx_t *s, idx_t n, idx_t k, std::vector<idx_t> &b, bool end)
{
    std::fill(b.begin(), b.end(), 0);
    for (idx_t i = 0; i < n; ++i) ++b[s[i]];
    idx_t sum = 0;
    for (idx_t c = 0; c < k; ++c) {
        sum += b[c];
        b[c] = end ? sum : sum - b[c];
    }
}

// L-type suffixes from the placed LMS ones (left to right), then S-type
// suffixes (right to left).
void induce(const idx_t *s, idx_t *sa, idx_t n, idx_t k, const std::vector<uint8_t> &stype, std::vector<idx_t> &b)
{
    bucket_bounds(s, n, k, b, false);
    for (idx_t i = 0; i < n; ++i) {
        const idx_t j = sa[i] - 1;
        if (sa[i] > 0 && !stype[j]) sa[b[s[j]]++] = j;
    }
    bucket_bounds(s, n, k, b, true);
    for (idx_t i = n - 1; i >= 0; --i) {
        const idx_t j = sa[i] - 1;
        if (sa[i] > 0 && stype[j]) sa[--b[s[j]]] = j;
    }
}

// s[0..n) over symbols 0..k-1 with s[n-1] = 0 the unique smallest (the
// sentinel); writes the suffix array to sa[0..n).
void sais(const idx_t *s, idx_t *sa, idx_t n, idx_t k)
{
    if (n == 1) {                                         // the terminator alone
        sa[0] = 0;
        return;
    }
    std::vector<uint8_t> stype((size_t)n);
    stype[n - 1] = 1;
    for (idx_t i = n - 2; i >= 0; --i)
        stype[i] = s[i] < s[i + 1] || (s[i] == s[i + 1] && stype[i + 1]);
    auto is_lms = [&](idx_t i) { return i > 0 && stype[i] && !stype[i - 1]; };
    std::vector<idx_t> b((size_t)k);

    // 1. LMS substrings in place at their bucket ends, then induced.
    std::fill(sa, sa + n, -1);
    bucket_bounds(s, n, k, b, true);
    for (idx_t i = 1; i < n; ++i)
        if (is_lms(i)) sa[--b[s[i]]] = i;
    induce(s, sa, n, k, stype, b);

    // 2. Compact the sorted LMS positions and name their substrings.
    idx_t m = 0;
    for (idx_t i = 0; i < n; ++i)
        if (is_lms(sa[i])) sa[m++] = sa[i];
    std::fill(sa + m, sa + n, -1);
    idx_t name = 0, prev = -1;
    for (idx_t t = 0; t < m; ++t) {
        const idx_t p = sa[t];
        bool diff = prev < 0;
        for (idx_t d = 0; !diff; ++d) {
            if (s[p + d] != s[prev + d] || stype[p + d] != stype[prev + d]) diff = true;
            else if (d > 0 && (is_lms(p + d) || is_lms(prev + d))) break;   // both substrings end here: equal
        }
        if (diff) {
            ++name;
            prev = p;
        }
        sa[m + p / 2] = name - 1;
    }
    // names of the LMS suffixes in text order form the reduced string
    idx_t j = n - 1;
    for (idx_t i = n - 1; i >= m; --i)
        if (sa[i] >= 0) sa[j--] = sa[i];
    idx_t *s1 = sa + n - m;
    idx_t *sa1 = sa;

    // 3. Sort the reduced string (directly when every name is unique).
    if (name < m) {
        sais(s1, sa1, m, name);
    } else {
        for (idx_t i = 0; i < m; ++i) sa1[s1[i]] = i;
    }

    // 4. Place the LMS suffixes in their sorted order and induce the rest.
    j = 0;
    for (idx_t i = 1; i < n; ++i)
        if (is_lms(i)) s1[j++] = i;                      // s1 now maps reduced index -> text position
    for (idx_t i = 0; i < m; ++i) sa1[i] = s1[sa1[i]];
    std::fill(sa + m, sa + n, -1);
    bucket_bounds(s, n, k, b, true);
    for (idx_t i = m - 1; i >= 0; --i) {
        const idx_t p = sa[i];
        sa[i] = -1;
        sa[--b[s[p]]] = p;
    }
    induce(s, sa, n, k, stype, b);
}

}  // namespace

extern "C" int bsw_sa_build(const uint8_t *codes, int64_t n, int32_t *sa)
{
    if (n < 0 || n >= INT32_MAX - 1 || (n > 0 && !codes) || !sa) return BSW_EINVAL;
    std::vector<idx_t> s;
    try {
        s.resize((size_t)n + 1);
    } catch (...) {
        return BSW_ENOMEM;
    }
    for (int64_t i = 0; i < n; ++i) {
        if (codes[i] > 3) return BSW_EINVAL;
        s[(size_t)i] = codes[i] + 1;                     // 1..4; 0 is the sentinel
    }
    s[(size_t)n] = 0;
    try {
        sais(s.data(), sa, (idx_t)n + 1, 5);
    } catch (const std::bad_alloc &) {
        return BSW_ENOMEM;
    }
    return BSW_OK;
}
