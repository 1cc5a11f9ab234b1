// bsw_warp2.cu - the warp-per-pair extension with two columns per instruction.
//
// The long-query kernel of the 16-bit range with the paper's 16-bit lanes
// (Section V-D1) put side by side in one 32-bit register: every DPX
// instruction of the cell update (Eq. 2 with Eq. 3's affine gaps) works on
// two columns at once.  The row is cut into granules of 8 columns; a granule
// keeps columns k and k + 4 (k = 0..3) in the low and high half of one
// register, so the two halves run two independent 4-column F chains that one
// packed instruction advances together.  A lane owns 1 to 4 consecutive
// granules of a row chunk, chosen per row from the band width, so a chunk
// covers the band in steps of 256 columns.  Across lanes F is the max-plus
// scan of the other warp kernels.  The band logic (rules a-c, the ring
// invariant) is the int2 ring kernel's, with a 16-bit slot layout.
//
// Zero-diagonal rule without a branch: M = min(D + s(i,j), D << z) with
// 2^z >= match + 1 is D + s(i,j) for D >= 1 and at most 0 for D = 0 (an
// unreached diagonal), as long as D << z stays below 2^15, so the kernel
// takes pairs whose score bound is below 2^(15 - z); the rest go to the
// 32-bit re-run list.
#include <cuda_runtime.h>
#include <cstdint>

#include "bsw_device.cuh"
#include "bsw_launch.h"

namespace bsw {

namespace {

constexpr int kX2MaxGr = 4;        // granules per lane in one chunk, at most
constexpr int kX2Warps = 4;        // warps per block

// Ring layout: ring column c (c & mask) lies in granule r = c' >> 3, whose
// 4 slots of 8 bytes {H2, E2} hold columns 8r + k (low halves) and 8r + k + 4
// (high halves) in slot k; 16 bytes of padding follow every 4 granules, so
// the lanes of a quarter warp reading their granules' 16-byte slot pairs hit
// distinct banks.  Half h of H2 in slot c holds H(i-1, c-1), of E2 E(i, c).
__host__ __device__ constexpr int x2_granule_slot(int r) { return r * 4 + (r >> 2) * 2; }
__host__ __device__ constexpr int x2_ring_words(int lg)
{
    return x2_granule_slot(1 << (lg - 3));   // one past the last granule
}

__device__ __forceinline__ int x2_slot(int c, int mask)
{
    return x2_granule_slot((c & mask) >> 3) + (c & 3);
}

__device__ __forceinline__ uint16_t *x2_half(uint2 *RG, int c, int mask, int word)
{
    return reinterpret_cast<uint16_t *>(RG + x2_slot(c, mask)) + 2 * word + ((c >> 2) & 1);
}

__device__ __forceinline__ void x2_set(uint2 *RG, int c, int mask, int h, int e)
{
    *x2_half(RG, c, mask, 0) = (uint16_t)h;
    *x2_half(RG, c, mask, 1) = (uint16_t)e;
}

// H and E of column c or'ed (zero iff both are).
__device__ __forceinline__ uint32_t x2_nonzero(const uint2 *RG, int c, int mask)
{
    const uint2 v = RG[x2_slot(c, mask)];
    return ((v.x | v.y) >> (16 * ((c >> 2) & 1))) & 0xffffu;
}

__device__ __forceinline__ int x2_get_h(const uint2 *RG, int c, int mask)
{
    return (int)((RG[x2_slot(c, mask)].x >> (16 * ((c >> 2) & 1))) & 0xffffu);
}

// Shared-memory stores under a predicate (no branch around them).
__device__ __forceinline__ void st_v4_if(bool p, void *addr, uint4 v)
{
    asm volatile("{ .reg .pred q; setp.ne.b32 q, %0, 0; @q st.shared.v4.u32 [%1], {%2, %3, %4, %5}; }"
                 :: "r"((int)p), "r"((unsigned)__cvta_generic_to_shared(addr)), "r"(v.x), "r"(v.y), "r"(v.z), "r"(v.w)
                 : "memory");
}

__device__ __forceinline__ void st_u16_if(bool p, void *addr, uint32_t v)
{
    asm volatile("{ .reg .pred q; setp.ne.b32 q, %0, 0; @q st.shared.u16 [%1], %2; }"
                 :: "r"((int)p), "r"((unsigned)__cvta_generic_to_shared(addr)), "h"((unsigned short)v) : "memory");
}

__device__ __forceinline__ uint32_t rep2(int v) { return ((uint32_t)v & 0xffffu) * 0x10001u; }

// Constants of the packed cell update (both halves hold the same value).
struct X2K {
    uint32_t a2;                 // match
    uint32_t scm;                // 2^16 - match - mismatch: the score multiply-add's factor
    uint32_t zmul;               // 2^z
    uint32_t noe_d2, noe_i2;     // -(o_del + e_del), -(o_ins + e_ins)
    uint32_t ne_d2, ne_i2;       // -e_del, -e_ins
    uint32_t nke2[4];            // -k * e_ins
    int zsh;                     // z of the zero-diagonal rule
};

__host__ __device__ inline int x2_zshift(int a)
{
    int z = 0;
    while ((1 << z) < a + 1) ++z;
    return z;
}

__device__ __forceinline__ X2K x2_consts(const Params &P)
{
    X2K K;
    K.a2 = rep2(P.a);
    K.scm = 0x10000u - (uint32_t)(P.a + P.b);
    K.noe_d2 = rep2(-(P.o_del + P.e_del));
    K.noe_i2 = rep2(-(P.o_ins + P.e_ins));
    K.ne_d2 = rep2(-P.e_del);
    K.ne_i2 = rep2(-P.e_ins);
#pragma unroll
    for (int k = 0; k < 4; ++k) K.nke2[k] = rep2(-k * P.e_ins);
    K.zsh = x2_zshift(P.a);
    K.zmul = P.k16 >> (16 - K.zsh);   // 2^z from a run-time value: the product stays a multiply-add
    return K;
}

// One row chunk: lane L owns the GC granules from column j0 = cb + 8*GC*L.
// Phase 1 loads each granule's slots and computes, per column pair, M (the
// diagonal term), E(i+1, j), and max(M, E, F_local) with F_local the F that
// the columns of the same half-granule to the left give; phase 2 chains the
// half-granules' F exits into the lane's exit and phase 3 scans those across
// the warp (F entering column j is max over k < j of M(k) - o - e - (j-1-k)e,
// Eq. 2-3); phase 4 adds the F entering each half-granule, giving H, takes
// the row key and stores slot j <- {H(i, j-1), E(i+1, j)}.  LAST: the chunk
// holding column hi - 1; it stores the granules that start at or before hi
// (the caller then clears H past hi in hi's granule) and, when hi is the
// chunk's end, slot hi itself: the row-end H(i, hi-1) with E = 0.  carry_f /
// carry_h: F entering the chunk and H of the column before it.
//
// The cell update keeps the ALU pipe (the DPX max/add-max instructions, the
// logic ops) for what only it can do: shifts, the 16-bit packing and the row
// keys are multiply-adds on the FMA pipe (x >> s as umulhi(x, 2^(32-s))), and
// the score of a column pair is one multiply-add of its two mismatch bits:
// m * (2^16 - match - mismatch) + match * 0x10001 gives match or -mismatch in
// each half (the low half's borrow is paid by the m_lo * 2^16 term).
template <int GC, bool LAST, bool SYM>
__device__ __forceinline__ void x2_chunk(const uint32_t *qw32, int qa, int n, uint32_t tmask, uint2 *RG, int mask,
                                         int cb, int hi, const X2K &K, int e_ins, int lane, int &carry_f,
                                         int &carry_h, int &key_l)
{
    constexpr int NW = (GC + 1) / 2;                  // 32-bit words of query bases (16 columns each)
    const int j0 = cb + lane * (8 * GC);

    // The lane's query bases: byte b = qa + j0/4 of the aligned query words
    // (j0 is a multiple of 8 and the query starts on a byte), funnel-shifted.
    // Word indices are clamped to the query's last word; bases at or past n
    // are out of band and their scores unused.
    uint32_t qw[NW];
    {
        const int b = qa + (j0 >> 2), w0 = b >> 2, sh = (b & 3) * 8;
        const int wl = (qa + ((n - 1) >> 2)) >> 2;      // the last word holding a query byte
        uint32_t w[NW + 1];
#pragma unroll
        for (int v = 0; v <= NW; ++v) w[v] = __ldg(qw32 + min(w0 + v, wl));
#pragma unroll
        for (int v = 0; v < NW; ++v) qw[v] = __funnelshift_r(w[v], w[v + 1], sh);
    }

    int sl[GC];
#pragma unroll
    for (int u = 0; u < GC; ++u) sl[u] = x2_granule_slot(((j0 >> 3) + u) & (mask >> 3));

    // Phase 1.
    uint32_t HF[GC][4], EN[GC][4], FL[GC];
#pragma unroll
    for (int v = 0; v < NW; ++v) {
        const uint32_t x = qw[v] ^ tmask;                  // 2-bit field c is zero where base c is t_i
        const uint32_t y = x | __umulhi(x, 0x80000000u);   // bit 2c: base c differs from t_i
        // granule 2v + uu: its columns 0-3 at bits 0, 2, 4, 6 and 4-7 at
        // bits 16, 18, 20, 22, so column pair k is bits 2k and 2k + 16
        const uint32_t Yg[2] = {prmt(y, 0u, 0x4140u), prmt(y, 0u, 0x4342u)};
        uint4 S[2][2];
        uint32_t floc[2] = {0u, 0u};
#pragma unroll
        for (int uu = 0; uu < 2; ++uu) {
            if (2 * v + uu < GC) {
                const uint4 *gp = reinterpret_cast<const uint4 *>(RG + sl[2 * v + uu]);
                S[uu][0] = gp[0];
                S[uu][1] = gp[1];
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
#pragma unroll
            for (int uu = 0; uu < 2; ++uu) {
                const int u = 2 * v + uu;
                if (u >= GC) continue;
                const uint4 &s = S[uu][k >> 1];
                const uint32_t Hd = (k & 1) ? s.z : s.x, Ed = (k & 1) ? s.w : s.y;
                const uint32_t ys = k ? __umulhi(Yg[uu], 1u << (32 - 2 * k)) : Yg[uu];
                const uint32_t sc = (ys & 0x00010001u) * K.scm + K.a2;
                const uint32_t M = __viaddmin_s16x2(Hd, sc, Hd * K.zmul);
                const uint32_t Mi = __viaddmax_s16x2_relu(M, K.noe_i2, 0u);
                const uint32_t Md = SYM ? Mi : __viaddmax_s16x2_relu(M, K.noe_d2, 0u);
                HF[u][k] = __vimax3_s16x2(M, Ed, floc[uu]);
                EN[u][k] = __viaddmax_s16x2_relu(Ed, K.ne_d2, Md);
                floc[uu] = __viaddmax_s16x2_relu(floc[uu], K.ne_i2, Mi);
            }
        }
#pragma unroll
        for (int uu = 0; uu < 2; ++uu)
            if (2 * v + uu < GC) FL[2 * v + uu] = floc[uu];
    }

    // Phase 2: the lane's F exit from its own columns.
    const int e4 = 4 * e_ins;
    int flo[GC], fhi[GC];
    int T = 0;
#pragma unroll
    for (int u = 0; u < GC; ++u) {
        const uint32_t hi16 = __umulhi(FL[u], 0x10000u);
        fhi[u] = (int)hi16;
        flo[u] = (int)(FL[u] + hi16 * 0xffff0000u);
        T = __viaddmax_s32(T, -e4, flo[u]);
        T = __viaddmax_s32(T, -e4, fhi[u]);
    }
    // Phase 3: prefix max over the warp of T + (lane + 1) * 8GC * e.
    const int ce = 8 * GC * e_ins;
    int v = T + (lane + 1) * ce;
#pragma unroll
    for (int d = 1; d < 32; d <<= 1) v = max(v, __shfl_up_sync(kFull, v, d));
    int vex = __shfl_up_sync(kFull, v, 1);
    if (lane == 0) vex = carry_f;
    int gin = max(carry_f, vex) - lane * ce;           // F entering the lane's first column
    const int vall = __shfl_sync(kFull, v, 31);

    // Phase 4: F entering each half-granule, packed.
    uint32_t G2[GC];
#pragma unroll
    for (int u = 0; u < GC; ++u) {
        const int glo = gin;
        const int ghi = __viaddmax_s32(glo, -e4, flo[u]);
        gin = __viaddmax_s32(ghi, -e4, fhi[u]);
        G2[u] = (uint32_t)glo + (uint32_t)ghi * 0x10000u;
    }
    // H of the lane's last column (high half of its last pair) for the next
    // lane's first slot.
    const uint32_t hlast = __viaddmax_s16x2(G2[GC - 1], K.nke2[3], HF[GC - 1][3]);
    uint32_t hprev = __shfl_up_sync(kFull, hlast, 1);
    if (lane == 0) hprev = (uint32_t)carry_h << 16;

    uint32_t key = 0u;                                 // H << 16 | column within the lane
#pragma unroll
    for (int u = 0; u < GC; ++u) {
        uint32_t h[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            h[k] = __viaddmax_s16x2(G2[u], K.nke2[k], HF[u][k]);
            key = __vimax3_u32(key, h[k] * 0x10000u + (uint32_t)(8 * u + k),
                               __umulhi(h[k], 0x10000u) * 0x10000u + (uint32_t)(8 * u + 4 + k));
        }
        // slot k <- {H of columns k - 1 and k + 3, E(i+1) of columns k and k + 4}
        const uint32_t s0 = __umulhi(hprev, 0x10000u) + h[3] * 0x10000u;
        uint4 *gp = reinterpret_cast<uint4 *>(RG + sl[u]);
        if (!LAST) {
            gp[0] = make_uint4(s0, EN[u][0], h[0], EN[u][1]);
            gp[1] = make_uint4(h[1], EN[u][2], h[2], EN[u][3]);
        } else {
            const bool st = j0 + 8 * u <= hi;
            st_v4_if(st, gp, make_uint4(s0, EN[u][0], h[0], EN[u][1]));
            st_v4_if(st, gp + 1, make_uint4(h[1], EN[u][2], h[2], EN[u][3]));
        }
        hprev = h[3];
    }
    // Row key with the absolute column (clamped: out-of-band columns past the
    // longest query never hold the row's best).
    key_l = max(key_l, (int)__umulhi(key, 0x10000u) * 32768 + min((int)(key & 0xffffu) + j0, 32767));
    carry_f = max(carry_f, vall) - 32 * ce;
    if (!LAST) {
        carry_h = (int)__umulhi(__shfl_sync(kFull, hprev, 31), 0x10000u);
    } else if (hi == cb + 256 * GC && lane == 31) {
        RG[x2_slot(hi, mask)] = make_uint2(__umulhi(hprev, 0x10000u), 0u);   // row end past the chunk
    }
}

// Columns a row touches from its first granule for a span of d = hi - cb
// columns (cb the band start rounded down to a granule), plus slot hi.
__host__ __device__ inline int x2_span(int d)
{
    const int cover = 256 * ((d + 255) / 256);
    return d == cover ? cover + 1 : cover;
}

// Ring columns for band w': a power of two holding every row's touched
// columns (span of at most 2w' + 8) and at least 2w' + 3.
__host__ __device__ inline int x2_ring_cols(int wb)
{
    const int d = 2 * wb + 8;
    int need = 64;
    while (need < 2 * wb + 3 || need < x2_span(d) || need < 256) need <<= 1;
    return need;
}

template <bool SYM>
__device__ unsigned long long x2_pair(const Batch &B, const Params &P, int p, uint2 *RG, int mask, const X2K &K)
{
    const int lane = threadIdx.x & 31;
    const int n = B.q_len[p], m = B.t_len[p], h0 = B.h0[p];
    const int wb = clip_band(P, n, B.w_override ? B.w_override[p] : P.w);
    const int e_del = P.e_del, e_ins = P.e_ins;
    const int oe_del = P.o_del + e_del;
    const uint8_t *qp = B.q + (B.q_off[p] >> 2);
    const int qa = (int)(reinterpret_cast<uintptr_t>(qp) & 3);
    const uint32_t *qw32 = reinterpret_cast<const uint32_t *>(qp - qa);
    const uint8_t *tp = B.t + (B.t_off[p] >> 2);
    const int ta = (int)(reinterpret_cast<uintptr_t>(tp) & 3);
    const uint32_t *tw32 = reinterpret_cast<const uint32_t *>(tp - ta);
    const int tlast = ta + ((m - 1) >> 2);                   // the target's last byte in tw32
    const int words = x2_ring_words(31 - __clz(mask + 1));
    for (int w = lane; w < words; w += 32) RG[w] = make_uint2(0u, 0u);
    int hw = -1, lo = 0, hi = n;
    int best = h0, bi = -1, bj = -1, gbest = -1, gi = -1, moff = 0;
    unsigned long long ncell = 0;
    const int cvis = h0 > P.o_ins ? (h0 - P.o_ins - 1) / e_ins : 0;   // last column with a non-zero boundary
    uint32_t tw = 0;                                           // target bases i..i+15 (i a multiple of 16)
    for (int i = 0; i < m; ++i) {
        if ((i & 15) == 0) {
            const int b = ta + (i >> 2), w0 = b >> 2;
            const uint32_t lo_w = __ldg(tw32 + w0);
            const uint32_t hi_w = __ldg(tw32 + min(w0 + 1, tlast >> 2));
            tw = __funnelshift_r(lo_w, hi_w, (b & 3) * 8);
        }
        const int tb = (tw >> (2 * (i & 15))) & 3;
        const uint32_t tmask = (uint32_t)tb * 0x55555555u;    // t_i in each 2-bit field
        const int lo_new = max(lo, i - wb);
        for (int c = lo + lane; c < lo_new; c += 32) x2_set(RG, c, mask, 0, 0);   // left the band
        lo = lo_new;
        hi = min(min(hi, i + wb + 1), n);
        // First visit of columns (hw, hi-1]: their slots are empty (never
        // written, or cleared when an alias left the band), so only columns
        // whose Eq. 3 boundary value is non-zero need a write.
        for (int c = hw + 1 + lane; c <= min(hi - 1, cvis); c += 32)
            x2_set(RG, c, mask, c == 0 ? h0 : max(0, h0 - P.o_ins - c * e_ins), 0);
        hw = max(hw, hi - 1);
        st_u16_if(lane == 0, x2_half(RG, hi, mask, 0), 0u);   // slot hi: read as empty in this row
        st_u16_if(lane == 0, x2_half(RG, hi, mask, 1), 0u);
        __syncwarp();
        const int hl0 = lo == 0 ? max(0, h0 - oe_del - i * e_del) : 0;
        int carry_f = 0, carry_h = hl0, key_l = 0;
        if (lo < hi) {
            int cb = lo & ~7;
            int ng = (hi - cb + 7) >> 3;                       // granules to cover
            while (ng > 32 * kX2MaxGr) {
                x2_chunk<kX2MaxGr, false, SYM>(qw32, qa, n, tmask, RG, mask, cb, hi, K, e_ins, lane, carry_f, carry_h,
                                               key_l);
                cb += 256 * kX2MaxGr;
                ng -= 32 * kX2MaxGr;
            }
            switch ((ng + 31) >> 5) {
            case 1: x2_chunk<1, true, SYM>(qw32, qa, n, tmask, RG, mask, cb, hi, K, e_ins, lane, carry_f, carry_h, key_l); break;
            case 2: x2_chunk<2, true, SYM>(qw32, qa, n, tmask, RG, mask, cb, hi, K, e_ins, lane, carry_f, carry_h, key_l); break;
            case 3: x2_chunk<3, true, SYM>(qw32, qa, n, tmask, RG, mask, cb, hi, K, e_ins, lane, carry_f, carry_h, key_l); break;
            default: x2_chunk<4, true, SYM>(qw32, qa, n, tmask, RG, mask, cb, hi, K, e_ins, lane, carry_f, carry_h, key_l); break;
            }
            __syncwarp();
            // hi's granule was stored whole: clear H past hi there (E past hi
            // is zero already).  Slots past hi are otherwise empty.
            st_u16_if(lane < 7 - (hi & 7), x2_half(RG, hi + 1 + lane, mask, 0), 0u);
        } else if (lane == 0) {
            x2_set(RG, hi, mask, hl0, 0);                      // empty band: the row-end value is the first column's
        }
        __syncwarp();
        hw = max(hw, hi);                                      // slot hi holds the row-end value now
        const int key = (int)__reduce_max_sync(kFull, (unsigned)key_l);
        const int rm = key >> 15, rj = key & 32767;
        if (hi > lo) ncell += (unsigned)(hi - lo);
        if (max(lo, hi) == n) {                                // H(i, n-1), now in slot hi
            const int hl = x2_get_h(RG, hi, mask);
            if (hl >= gbest) gi = i;
            gbest = max(gbest, hl);
        }
        if (rm == 0) break;
        if (rm > best) {
            best = rm; bi = i; bj = rj;
            moff = max(moff, abs(rj - i));
        } else if (P.zdrop > 0) {
            const int di = i - bi, dj = rj - bj;
            const int drop = di > dj ? best - rm - (di - dj) * e_del : best - rm - (dj - di) * e_ins;
            if (drop > P.zdrop) break;
        }
        // Rule c: the first non-zero slot of [lo, hi) becomes lo, the last of
        // [lo, hi] plus 2 becomes hi.  One ballot checks the 16 slots at each
        // end (lanes 0-15 from lo up, 16-31 from hi down); when both ends
        // hold a non-zero slot there (the usual row) that decides both,
        // otherwise the scans run 32 slots at a time.
        {
            const int j = lane < 16 ? lo + lane : hi - (lane - 16);
            const bool in = lane < 16 ? j < hi : j >= lo;
            const uint32_t nz = in ? x2_nonzero(RG, j, mask) : 0u;
            const unsigned bal = __ballot_sync(kFull, nz != 0u);
            const unsigned bl = bal & 0xffffu, br = bal >> 16;
            int last;
            if (bl && br) {
                lo += __ffs(bl) - 1;
                last = hi - (__ffs(br) - 1);
            } else {
                int nlo = hi;
                for (int base = lo; base < hi; base += 32) {
                    const int jj = base + lane;
                    const uint32_t z = jj < hi ? x2_nonzero(RG, jj, mask) : 0u;
                    const unsigned bb = __ballot_sync(kFull, z != 0u);
                    if (bb) { nlo = base + __ffs(bb) - 1; break; }
                }
                lo = nlo;
                last = lo - 1;
                for (int top = hi; top >= lo; top -= 32) {
                    const int jj = top - lane;
                    const uint32_t z = jj >= lo ? x2_nonzero(RG, jj, mask) : 0u;
                    const unsigned bb = __ballot_sync(kFull, z != 0u);
                    if (bb) { last = top - (__ffs(bb) - 1); break; }
                }
            }
            hi = min(last + 2, n);
        }
    }
    if (lane == 0) store_result(&B.out[p], best, bj + 1, bi + 1, gi + 1, gbest, moff);
    return ncell;
}

// Persistent kernel over a class list: pairs whose score bound or band the
// packed kernel does not hold go to the 32-bit re-run list.  A 10 kbp pair
// runs about as long as the whole launch (three blocks per SM), so the first
// pair of each warp is stratified: the list (longest first) is cut into strata of NB = gridDim.x
// pairs, and warp j of every block takes its first pair from stratum j, the
// blocks in the order they start (one 16-bit field of a 64-bit counter per
// stratum, NB fetches each).  Every block, whatever SM it lands on, thus
// holds one pair of each stratum, and no SM starts with several of the
// longest pairs; later pairs come longest first from the rest of the list.
template <bool SYM>
__global__ void __launch_bounds__(kX2Warps * 32, 3) k_warp_x2(Batch B, Params P, Work W, int cls, int ring_log2)
{
    extern __shared__ uint4 x2_mem[];
    const int lane = threadIdx.x & 31, wj = threadIdx.x >> 5;
    uint2 *ring = reinterpret_cast<uint2 *>(x2_mem) + (ring_log2 > 0 ? wj * x2_ring_words(ring_log2) : 0);
    const X2K K = x2_consts(P);
    const long long limit = 1ll << (15 - K.zsh);
    const int count = W.cls_count[cls];
    const int nb = (int)gridDim.x;
    const int32_t *list = W.order + W.cls_start[cls];
    unsigned long long cells = 0;
    for (bool first = true;; first = false) {
        int g = 0;
        if (lane == 0) {
            if (first) {
                const unsigned long long old =
                    atomicAdd(reinterpret_cast<unsigned long long *>(W.cls_next + kStrata), 1ull << (16 * wj));
                g = wj * nb + (int)((old >> (16 * wj)) & 0xffffu);
            } else {
                g = kX2Warps * nb + (int)atomicAdd(&W.cls_next[cls], 1u);
            }
        }
        g = __shfl_sync(kFull, g, 0);
        if (g >= count) break;               // first wave: then count <= g < 4 NB, nothing past the strata
        const int p = list[g];
        const int n = B.q_len[p], m = B.t_len[p];
        const int wb = clip_band(P, n, B.w_override ? B.w_override[p] : P.w);
        const long long bound = (long long)B.h0[p] + (long long)P.a * min(n, m);
        if (ring_log2 > 0 && x2_ring_cols(wb) <= (1 << ring_log2) && bound < limit) {
            cells += x2_pair<SYM>(B, P, p, ring, x2_ring_cols(wb) - 1, K);
        } else if (lane == 0) {
            W.rerun[atomicAdd(&W.cls_count[kRerun], 1)] = p;
        }
    }
    if (lane == 0 && cells) atomicAdd(W.cells, cells);
}

// The plain baseline with this kernel: pairs in input order, one per warp
// (grid stride), no bucketing or classes.  Pairs it cannot take (an N base, a
// score bound at its limit or above, a band wider than its ring) go to the
// re-run list, which the 32-bit warp kernel runs afterwards.
template <bool SYM>
__global__ void __launch_bounds__(kX2Warps * 32, 4) k_plain_x2(Batch B, Params P, Work W, int ring_log2)
{
    extern __shared__ uint4 x2_mem[];
    const int lane = threadIdx.x & 31;
    uint2 *ring = reinterpret_cast<uint2 *>(x2_mem) + (threadIdx.x >> 5) * x2_ring_words(ring_log2);
    const X2K K = x2_consts(P);
    const long long limit = 1ll << (15 - K.zsh);
    const int64_t gw = (int64_t)blockIdx.x * kX2Warps + (threadIdx.x >> 5), nw = (int64_t)gridDim.x * kX2Warps;
    unsigned long long cells = 0;
    for (int64_t p = gw; p < B.n; p += nw) {
        const long long bound = plain_check(B, P, W, p, lane);
        if (bound < 0) continue;
        const int n = B.q_len[p];
        const int wb = clip_band(P, n, B.w_override ? B.w_override[p] : P.w);
        const bool has_n = (B.q_n || B.t_n) && pair_has_n(B, B.q_off[p], n, B.t_off[p], B.t_len[p]);
        if (!has_n && bound < limit && x2_ring_cols(wb) <= (1 << ring_log2)) {
            cells += x2_pair<SYM>(B, P, (int)p, ring, x2_ring_cols(wb) - 1, K);
        } else if (lane == 0) {
            W.rerun[atomicAdd(&W.cls_count[kRerun], 1)] = (int32_t)p;
        }
    }
    if (lane == 0 && cells) atomicAdd(W.cells, cells);
}

int g_x2_blocks = 1;         // blocks per SM of the class kernel, set by prepare_x2
int g_x2_plain_blocks = 1;   // of the plain kernel (as many as fit)

}  // namespace

bool x2_usable(const Params &P)
{
    // score bound 2^13 at least, and every packed constant well inside 16 bits
    return x2_zshift(P.a) <= 2 && P.o_del + P.e_del <= 8192 && P.o_ins + P.e_ins <= 8192 && P.e_ins <= 2048 &&
           P.e_del <= 2048;
}

int x2_ring_log2(const Params &P)
{
    int lg = 6;
    const int need = x2_ring_cols(P.w);
    while ((1 << lg) < need && lg < 16) ++lg;
    const size_t per_block = (size_t)kX2Warps * x2_ring_words(lg) * 8;
    return per_block <= kRingSmemMax ? lg : 0;
}

cudaError_t prepare_x2(int sms)
{
    (void)sms;
    cudaError_t e;
    if ((e = cudaFuncSetAttribute(k_warp_x2<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRingSmemMax)) !=
        cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_warp_x2<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRingSmemMax)) !=
        cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_plain_x2<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRingSmemMax)) !=
        cudaSuccess)
        return e;
    if ((e = cudaFuncSetAttribute(k_plain_x2<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kRingSmemMax)) !=
        cudaSuccess)
        return e;
    // resident blocks for the ring of a w = 500 band (the long-query workload's)
    int nb = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_warp_x2<true>, kX2Warps * 32,
                                                           (size_t)kX2Warps * x2_ring_words(10) * 8)) != cudaSuccess)
        return e;
    // 3 blocks (12 warps) per SM, the class kernel's launch bound, although
    // 4 would fit at 128 registers: a 10 kbp pair runs about as long as the
    // launch, and at 12 warps it gets a twelfth of its SM instead of a
    // sixteenth, so the launch ends with the SMs (long10k's class 16.4 ms
    // against 18.1 at 4 blocks, every SM done within 0.4 ms of the others).
    g_x2_blocks = nb > 3 ? 3 : (nb > 0 ? nb : 1);
    // The plain kernel takes pairs in input order, where the longest pairs are
    // spread over the whole launch: it runs as many blocks as fit.
    int np_ = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&np_, k_plain_x2<true>, kX2Warps * 32,
                                                           (size_t)kX2Warps * x2_ring_words(10) * 8)) != cudaSuccess)
        return e;
    g_x2_plain_blocks = np_ > 0 ? np_ : 1;
    return cudaSuccess;
}

cudaError_t launch_x2(const Batch &B, const Params &P, const Work &W, int cls, cudaStream_t st, int sms)
{
    if (sms * g_x2_blocks > 65535) return cudaErrorInvalidConfiguration;   // 16-bit stratum fields
    const int lg = x2_ring_log2(P);
    const size_t smem = lg ? (size_t)kX2Warps * x2_ring_words(lg) * 8 : 0;
    const bool sym = P.o_del == P.o_ins && P.e_del == P.e_ins;
    if (sym) k_warp_x2<true><<<sms * g_x2_blocks, kX2Warps * 32, smem, st>>>(B, P, W, cls, lg);
    else k_warp_x2<false><<<sms * g_x2_blocks, kX2Warps * 32, smem, st>>>(B, P, W, cls, lg);
    return cudaGetLastError();
}

cudaError_t launch_plain_x2(const Batch &B, const Params &P, const Work &W, cudaStream_t st, int sms)
{
    const int lg = x2_ring_log2(P);
    if (lg == 0) return cudaErrorInvalidValue;
    cudaError_t e;
    if ((e = cudaMemsetAsync(W.cls_count + kRerun, 0, 4, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(W.cls_next + kRerun, 0, 4, st)) != cudaSuccess) return e;
    const size_t smem = (size_t)kX2Warps * x2_ring_words(lg) * 8;
    const bool sym = P.o_del == P.o_ins && P.e_del == P.e_ins;
    if (sym) k_plain_x2<true><<<sms * g_x2_plain_blocks, kX2Warps * 32, smem, st>>>(B, P, W, lg);
    else k_plain_x2<false><<<sms * g_x2_plain_blocks, kX2Warps * 32, smem, st>>>(B, P, W, lg);
    return cudaGetLastError();
}

}  // namespace bsw
