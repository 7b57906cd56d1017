// Near field of the FMM (Section 3.7, A^(sparse) X) and the direct all-pairs product
// (Section 3.9, brute force), both with the one-point quadrature kernel of Eq. (ns1):
//   u_i += sum_{j != i} [ q_j / |r_i - r_j| + w_j n_j.(r_i - r_j) / |r_i - r_j|^3 ],
// q_j = f s_j X_L,j / (4 pi), w_j = g s_j X_M,j / (4 pi) (Eqs. (2.13), (3.27)).
//
// FP32 variants keep coordinates accurate by construction: the list kernel works in
// leaf-box units with coordinates relative to each leaf centre (integer box offsets are
// exact in FP32), the direct kernel splits coordinates into hi + lo FP32 pairs. Sums are
// formed per shared-memory tile in FP32 and merged with TwoSum compensation.
//
// The single-layer kernel of Eq. (ns1) is symmetric in r = |r_i - r_j|, so the FP32 single-RHS,
// single-layer products (every GMRES product) evaluate every pair of neighbour leaves A < B
// once, by A's units: one reciprocal square root feeds both q_j / r into r_i and q_i / r into
// r_j. B's shares are summed over A's receivers inside the warp, stored per (unit of A, B), and
// added to B's points by a second kernel in a fixed order: no atomics, deterministic results.
// Products with the double layer run one way: its exchanged dipole term (n_i instead of n_j)
// costs more arithmetic and registers than the shared square root saves (measured: 5.96 ms
// symmetric against 5.37 ms one way at the benchmark's size).
#include "internal.h"

#include <algorithm>
#include <type_traits>

namespace bem {
namespace {

constexpr int P2P_THREADS = 128;
constexpr double kInv4Pi = 0.0795774715459476678844418816862571810;

template <class T>
__device__ __forceinline__ T rsqrt_t(T x);
// The hardware approximation (relative error below 2^-22) without the denormal handling of
// rsqrtf: r^2 is never denormal here (coordinates are in leaf-box units), and r^2 = 0 gives
// +inf, which the self-pair test replaces by 0.
template <>
__device__ __forceinline__ float rsqrt_t<float>(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
template <>
__device__ __forceinline__ double rsqrt_t<double>(double x) { return rsqrt(x); }

template <class T>
struct Comp {
    T s = 0, c = 0;
    __device__ __forceinline__ void add(T v) {
        T t = s + v;
        T bp = t - s;
        c += (s - (t - bp)) + (v - bp);
        s = t;
    }
    __device__ __forceinline__ double get() const { return (double)s + (double)c; }
};

template <class T>
struct V4 {
    using type = float4;
};
template <>
struct V4<double> {
    using type = double4;
};

// Near-field work is split into units of up to 64 receivers of one leaf (Tree::p2p_units);
// one warp owns a unit and each lane keeps two receivers in registers, so a staged source feeds
// two pairs; a unit of fewer receivers splits each source tile over groups of lanes instead of
// leaving lanes idle. The warp
// walks the (up to 27) neighbour leaves; each neighbour's sources are staged 32 at a time in
// the warp's own shared-memory slice as (x, y, z, q) and (n_x, n_y, n_z, w), positions
// relative to the target leaf's centre in leaf-box units. HQ / HW select the single- and
// double-layer terms, so a product with one layer only (every GMRES product) pays for that
// layer alone. The self pair has r^2 = 0 exactly (same coordinates, zero offset) and is
// skipped; only the target leaf's own tiles can hold it, so only they test r^2 (the paper's
// quadrature excludes j = i, Eq. (ns1); distinct vertices never coincide on a valid mesh).
constexpr int P2P_WARPS = 4;   // warps (work units) per block
constexpr int P2P_UNIT = 64;   // receivers per work unit

template <class T, int R, bool HQ, bool HW>
struct P2PStage {
    using T4 = typename V4<T>::type;
    T4 a[32];                                  // x, y, z, q (first RHS)
    T4 b[HW ? 32 : 1];                         // n_x, n_y, n_z, w (first RHS)
    T q[(R > 1 && HQ) ? R - 1 : 1][32];        // q of the other RHS
    T w[(R > 1 && HW) ? R - 1 : 1][32];        // w of the other RHS
};

template <class T, int R, int KR, bool HQ, bool HW, bool SELF>
__device__ __forceinline__ void p2p_source(const P2PStage<T, R, HQ, HW> &sg, int s, const T *xi, const T *yi,
                                           const T *zi, T (*part)[R]) {
    using T4 = typename V4<T>::type;
    const T4 a = sg.a[s];
    T4 bb;
    if (HW) bb = sg.b[s];
#pragma unroll
    for (int k = 0; k < KR; ++k) {
        const T dx = xi[k] - a.x, dy = yi[k] - a.y, dz = zi[k] - a.z;
        const T r2 = dx * dx + dy * dy + dz * dz;
        const T rinv = SELF ? (r2 > (T)0 ? rsqrt_t<T>(r2) : (T)0) : rsqrt_t<T>(r2);
        if (HQ) {
            part[k][0] += a.w * rinv;
#pragma unroll
            for (int r = 1; r < R; ++r) part[k][r] += sg.q[r - 1][s] * rinv;
        }
        if (HW) {
            const T nd3 = (bb.x * dx + bb.y * dy + bb.z * dz) * (rinv * rinv * rinv);
            part[k][0] += bb.w * nd3;
#pragma unroll
            for (int r = 1; r < R; ++r) part[k][r] += sg.w[r - 1][s] * nd3;
        }
    }
}

// One staged tile of up to 32 sources against a lane's two receivers. The warp's lanes form G
// groups of 32/G lanes; group gi takes the sources gi * 32/G .. (gi + 1) * 32/G - 1 of the tile,
// so a unit of few receivers still keeps every lane busy (its groups' partial sums are merged
// at the end of the unit).
template <class T, int R, int G, bool HQ, bool HW, bool SELF>
__device__ __forceinline__ void p2p_tile(const P2PStage<T, R, HQ, HW> &sg, int ns, int gi, const T *xi, const T *yi,
                                         const T *zi, Comp<T> (*acc)[R]) {
    constexpr int SG = 32 / G;  // sources per group and tile
    T part[2][R];
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int r = 0; r < R; ++r) part[k][r] = (T)0;
    const int s0 = gi * SG;
    if (ns == 32) {  // full tile: fixed trip count
#pragma unroll 8
        for (int t = 0; t < SG; ++t) p2p_source<T, R, 2, HQ, HW, SELF>(sg, s0 + t, xi, yi, zi, part);
    } else {
        const int e = min(SG, ns - s0);  // may be <= 0 for the groups past the tile's end
#pragma unroll 2
        for (int t = 0; t < e; ++t) p2p_source<T, R, 2, HQ, HW, SELF>(sg, s0 + t, xi, yi, zi, part);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int r = 0; r < R; ++r) acc[k][r].add(part[k][r]);
}

// One work unit (up to 64 receivers of one leaf) by one warp, its lanes split into G groups
// (G = 1 for 33..64 receivers, 2 for 17..32, 4 for 9..16, 8 for 1..8): lane = gi * (32/G) + rs
// holds the receivers rs and rs + 32/G and takes group gi's share of every source tile.
template <class T, int R, int G, bool HQ, bool HW>
__device__ __forceinline__ void p2p_unit_g(P2PStage<T, R, HQ, HW> &sg, int lane, int b, int r0, int nr,
                                           const int32_t *__restrict__ bstart, const int32_t *__restrict__ bcount,
                                           const int32_t *__restrict__ nbr, const int32_t *__restrict__ ncnt,
                                           const int8_t *__restrict__ nd, int64_t N, const T *__restrict__ loc,
                                           const T *__restrict__ nrm, const T *__restrict__ q, const T *__restrict__ w,
                                           double *__restrict__ out) {
    constexpr int LG = 32 / G;  // lanes per group
    const int rs = lane & (LG - 1), gi = lane / LG;
    const int s0 = bstart[b];
    T xi[2], yi[2], zi[2];
    Comp<T> acc[2][R];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int li = rs + k * LG;
        const int64_t i = s0 + r0 + (li < nr ? li : 0);
        xi[k] = loc[i];
        yi[k] = loc[N + i];
        zi[k] = loc[2 * N + i];
    }
    // neighbour table of the target leaf, one entry per lane, broadcast by shuffles
    const int nn = ncnt[b];
    int my_f = 0;
    T my_d[3] = {(T)0, (T)0, (T)0};
    if (lane < nn) {
        my_f = nbr[b * 27 + lane];
#pragma unroll
        for (int d = 0; d < 3; ++d) my_d[d] = (T)nd[(b * 27 + lane) * 4 + d];
    }
    for (int k = 0; k < nn; ++k) {
        const int f = __shfl_sync(0xffffffffu, my_f, k);
        const T ox = __shfl_sync(0xffffffffu, my_d[0], k);
        const T oy = __shfl_sync(0xffffffffu, my_d[1], k);
        const T oz = __shfl_sync(0xffffffffu, my_d[2], k);
        const int fs = bstart[f], fc = bcount[f];
        const bool self = (f == b);
        for (int t0 = 0; t0 < fc; t0 += 32) {
            if (t0 + lane < fc) {
                const int64_t j = fs + t0 + lane;
                sg.a[lane] = typename V4<T>::type{loc[j] + ox, loc[N + j] + oy, loc[2 * N + j] + oz,
                                                  HQ ? q[j] : (T)0};
                if (HW) sg.b[lane] = typename V4<T>::type{nrm[j], nrm[N + j], nrm[2 * N + j], w[j]};
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    if (HQ) sg.q[r - 1][lane] = q[r * N + j];
                    if (HW) sg.w[r - 1][lane] = w[r * N + j];
                }
            }
            __syncwarp();
            const int ns = min(32, fc - t0);
            if (self) p2p_tile<T, R, G, HQ, HW, true>(sg, ns, gi, xi, yi, zi, acc);
            else p2p_tile<T, R, G, HQ, HW, false>(sg, ns, gi, xi, yi, zi, acc);
            __syncwarp();
        }
    }
    // merge the groups' partial sums into group 0 (a fixed butterfly: deterministic)
#pragma unroll
    for (int off = LG; off < 32; off <<= 1)
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const T os = __shfl_xor_sync(0xffffffffu, acc[k][r].s, off);
                const T oc = __shfl_xor_sync(0xffffffffu, acc[k][r].c, off);
                acc[k][r].add(os);
                acc[k][r].c += oc;
            }
    if (gi == 0) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int li = rs + k * LG;
            if (li < nr) {
                const int64_t i = s0 + r0 + li;
#pragma unroll
                for (int r = 0; r < R; ++r) out[r * N + i] = acc[k][r].get();  // the far field is added later
            }
        }
    }
}

template <class T, int R, bool HQ, bool HW>
__device__ __forceinline__ void p2p_unit(P2PStage<T, R, HQ, HW> &sg, int lane, int2 un,
                                         const int32_t *__restrict__ bstart, const int32_t *__restrict__ bcount,
                                         const int32_t *__restrict__ nbr, const int32_t *__restrict__ ncnt,
                                         const int8_t *__restrict__ nd, int64_t N, const T *__restrict__ loc,
                                         const T *__restrict__ nrm, const T *__restrict__ q, const T *__restrict__ w,
                                         double *__restrict__ out) {
    const int b = un.x, r0 = un.y;
    const int nr = min(P2P_UNIT, bcount[b] - r0);  // uniform in the warp
    if (nr > 32) p2p_unit_g<T, R, 1, HQ, HW>(sg, lane, b, r0, nr, bstart, bcount, nbr, ncnt, nd, N, loc, nrm, q, w, out);
    else if (nr > 16) p2p_unit_g<T, R, 2, HQ, HW>(sg, lane, b, r0, nr, bstart, bcount, nbr, ncnt, nd, N, loc, nrm, q, w, out);
    else if (nr > 8) p2p_unit_g<T, R, 4, HQ, HW>(sg, lane, b, r0, nr, bstart, bcount, nbr, ncnt, nd, N, loc, nrm, q, w, out);
    else p2p_unit_g<T, R, 8, HQ, HW>(sg, lane, b, r0, nr, bstart, bcount, nbr, ncnt, nd, N, loc, nrm, q, w, out);
}

// FP32 form with packed two-wide arithmetic (add/mul/fma .f32x2: one instruction for two
// lanes' worth of FP32 work). The near field is issue-bound, so each lane takes its two
// receivers against two sources at a time: a staged tile holds 16 source pairs, each as
// (-x, -x', -y, -y'), (-z, -z', q, q') (and (n_x, n_x', n_y, n_y'), (n_z, n_z', w, w') for the
// double layer); a receiver's coordinate is a broadcast pair, so x_i - x_j is one packed add of
// the negated source coordinate (exactly the scalar difference) and r^2, the sums and the
// double layer's n.(r_i - r_j) / r^3 are packed products; the reciprocal square roots stay
// scalar. Lanes past a tile's end stage a source of zero strength far outside the leaf's
// neighbourhood (finite r^2), so a partial tile runs whole pairs.
template <int R, bool HQ, bool HW>
struct P2PStageX2 {
    float4 a[16];               // -x, -x', -y, -y'
    float4 b[16];               // -z, -z', q, q' (first RHS)
    float4 c[HW ? 16 : 1];      // n_x, n_x', n_y, n_y'
    float4 d[HW ? 16 : 1];      // n_z, n_z', w, w' (first RHS)
    float q[(R > 1 && HQ) ? R - 1 : 1][32];
    float w[(R > 1 && HW) ? R - 1 : 1][32];
    float tr[R == 1 ? 32 : 1][20];  // symmetric form: per-lane rows of the sources' shares, transposed
};

template <bool SELF>
__device__ __forceinline__ float2 rsqrt_x2(float2 r2) {
    float2 ri;
    ri.x = SELF ? (r2.x > 0.f ? rsqrt_t<float>(r2.x) : 0.f) : rsqrt_t<float>(r2.x);
    ri.y = SELF ? (r2.y > 0.f ? rsqrt_t<float>(r2.y) : 0.f) : rsqrt_t<float>(r2.y);
    return ri;
}

// The receivers' own strengths for the symmetric form (broadcast pairs, zero for lanes past the
// unit's end).
struct RecvX2 {
    float2 q[2];
};

// BACK (single layer): also accumulate the pair's share for the two sources, the sum over this
// lane's receivers of q_i / r
template <int R, bool HQ, bool HW, bool SELF, bool BACK = false>
__device__ __forceinline__ void p2p_source_x2(const P2PStageX2<R, HQ, HW> &sg, int p, const float2 *X,
                                              const float2 *Y, const float2 *Z, float2 (*part)[R],
                                              const RecvX2 *rv = nullptr, float2 *bk = nullptr) {
    const float4 A = sg.a[p], B = sg.b[p];
    const float2 mx = make_float2(A.x, A.y), my = make_float2(A.z, A.w), mz = make_float2(B.x, B.y);
    float4 C, D;
    if (HW) {
        C = sg.c[p];
        D = sg.d[p];
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const float2 dx = __fadd2_rn(X[k], mx), dy = __fadd2_rn(Y[k], my), dz = __fadd2_rn(Z[k], mz);
        float2 r2 = __fmul2_rn(dx, dx);
        r2 = __ffma2_rn(dy, dy, r2);
        r2 = __ffma2_rn(dz, dz, r2);
        const float2 ri = rsqrt_x2<SELF>(r2);
        if (HQ) {
            part[k][0] = __ffma2_rn(make_float2(B.z, B.w), ri, part[k][0]);
#pragma unroll
            for (int r = 1; r < R; ++r)
                part[k][r] = __ffma2_rn(*reinterpret_cast<const float2 *>(&sg.q[r - 1][2 * p]), ri, part[k][r]);
            if (BACK) *bk = __ffma2_rn(rv->q[k], ri, *bk);
        }
        if (HW) {
            float2 nd = __fmul2_rn(make_float2(C.x, C.y), dx);
            nd = __ffma2_rn(make_float2(C.z, C.w), dy, nd);
            nd = __ffma2_rn(make_float2(D.x, D.y), dz, nd);
            const float2 nd3 = __fmul2_rn(nd, __fmul2_rn(__fmul2_rn(ri, ri), ri));
            part[k][0] = __ffma2_rn(make_float2(D.z, D.w), nd3, part[k][0]);
#pragma unroll
            for (int r = 1; r < R; ++r)
                part[k][r] = __ffma2_rn(*reinterpret_cast<const float2 *>(&sg.w[r - 1][2 * p]), nd3, part[k][r]);
        }
    }
}

// A staged tile of an owned neighbour leaf (symmetric form, one RHS): the forward sums as in
// p2p_tile_x2 and, per batch of up to 16 sources of a group, each source's share summed over the
// unit's receivers (every group holds all of them), written to back[s] for the tile's source s.
// The sum over lanes goes through shared memory: every lane stores its row of the batch's
// values, then lane rs adds up column rs over its group's rows (for one group of 32 lanes, each
// half of the warp takes half the rows and one shuffle joins them). The groups read their rows
// in skewed orders so that their columns fall in different banks; the order of every sum is
// fixed, so the result is deterministic.
template <int G, bool HQ, bool HW>
__device__ __forceinline__ void p2p_tile_x2_sym(P2PStageX2<1, HQ, HW> &sg, int ns, int gi, int lane,
                                                const float2 *X, const float2 *Y, const float2 *Z, const RecvX2 &rv,
                                                Comp<float> (*acc)[1], float *__restrict__ back) {
    constexpr int SP = 16 / G, LG = 32 / G;
    constexpr int HP = SP < 8 ? SP : 8;  // source pairs per batch
    constexpr int NV = 2 * HP;           // sources per batch: values per lane
    constexpr int SK = G == 2 ? 4 : (G == 4 ? 2 : 1);  // row skew per group (see above)
    const int rs = lane & (LG - 1);
    float2 part[2][1];
    part[0][0] = part[1][0] = make_float2(0.f, 0.f);
    const int p0 = gi * SP;
    const int e = min(SP, (ns + 1) / 2 - p0);  // pairs of this group holding sources
#pragma unroll
    for (int h0 = 0; h0 < SP; h0 += HP) {
        if (ns == 32) {
            float2 bk[HP];
#pragma unroll
            for (int t = 0; t < HP; ++t) bk[t] = make_float2(0.f, 0.f);
#pragma unroll
            for (int t = 0; t < HP; ++t) p2p_source_x2<1, HQ, HW, false, true>(sg, p0 + h0 + t, X, Y, Z, part, &rv, &bk[t]);
            float4 *row = reinterpret_cast<float4 *>(&sg.tr[lane][0]);
#pragma unroll
            for (int c4 = 0; c4 < NV / 4; ++c4)
                row[c4] = make_float4(bk[2 * c4].x, bk[2 * c4].y, bk[2 * c4 + 1].x, bk[2 * c4 + 1].y);
        } else {  // a partial tile: a rolled loop (small code), each pair's shares stored as it goes
#pragma unroll 1
            for (int t = 0; t < HP; ++t) {
                float2 b = make_float2(0.f, 0.f);
                if (h0 + t < e) p2p_source_x2<1, HQ, HW, false, true>(sg, p0 + h0 + t, X, Y, Z, part, &rv, &b);
                *reinterpret_cast<float2 *>(&sg.tr[lane][2 * t]) = b;
            }
        }
        __syncwarp();
        float tot = 0.f;
        if constexpr (G == 1) {
            const int half = lane >> 4, col = lane & 15;
#pragma unroll
            for (int r = 0; r < 16; ++r) tot += sg.tr[half * 16 + ((r + 4 * half) & 15)][col];
            tot += __shfl_xor_sync(0xffffffffu, tot, 16);
        } else {
            const int sk = G == 8 ? (gi >> 1) : SK * gi;
#pragma unroll
            for (int r = 0; r < LG; ++r) tot += sg.tr[gi * LG + ((r + sk) & (LG - 1))][rs];
        }
        __syncwarp();  // the next batch rewrites the rows
        const int src = 2 * (p0 + h0) + (rs & (NV - 1));
        if (rs < NV && src < ns) back[src] = tot;
    }
#pragma unroll
    for (int k = 0; k < 2; ++k) acc[k][0].add(part[k][0].x + part[k][0].y);
}

// one staged tile (up to 16 source pairs) against a lane's two receivers; group gi of G takes
// the pairs gi * 16/G .. (gi + 1) * 16/G - 1
template <int R, int G, bool HQ, bool HW, bool SELF>
__device__ __forceinline__ void p2p_tile_x2(const P2PStageX2<R, HQ, HW> &sg, int ns, int gi, const float2 *X,
                                            const float2 *Y, const float2 *Z, Comp<float> (*acc)[R]) {
    constexpr int SP = 16 / G;  // source pairs per group and tile
    float2 part[2][R];
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int r = 0; r < R; ++r) part[k][r] = make_float2(0.f, 0.f);
    const int p0 = gi * SP;
    if (ns == 32) {
#pragma unroll 4
        for (int t = 0; t < SP; ++t) p2p_source_x2<R, HQ, HW, SELF>(sg, p0 + t, X, Y, Z, part);
    } else {
        const int e = min(SP, (ns + 1) / 2 - p0);
#pragma unroll 1
        for (int t = 0; t < e; ++t) p2p_source_x2<R, HQ, HW, SELF>(sg, p0 + t, X, Y, Z, part);
    }
#pragma unroll
    for (int k = 0; k < 2; ++k)
#pragma unroll
        for (int r = 0; r < R; ++r) acc[k][r].add(part[k][r].x + part[k][r].y);
}

// Symmetric form (SYM, one RHS): a neighbour leaf f > b is owned: its tiles also produce the
// shares of f's points, written at back + back_unit + (owned points before f) + tile offset; a
// neighbour f < b is skipped (f's units evaluate the pair and b's points get their shares by
// the gather); the leaf's own tiles are evaluated one way, all pairs i != j.
struct BackArgs {
    float *back;
    const int32_t *S;
    const int64_t *base;
};

// the packed counterpart of p2p_unit_g (same units, lanes, groups and merge)
template <int R, int G, bool HQ, bool HW, bool SYM = false>
__device__ __forceinline__ void p2p_unit_gx2(P2PStageX2<R, HQ, HW> &sg, int lane, int b, int r0, int nr,
                                             const int32_t *__restrict__ bstart, const int32_t *__restrict__ bcount,
                                             const int32_t *__restrict__ nbr, const int32_t *__restrict__ ncnt,
                                             const int8_t *__restrict__ nd, int64_t N, const float *__restrict__ loc,
                                             const float *__restrict__ nrm, const float *__restrict__ q,
                                             const float *__restrict__ w, double *__restrict__ out,
                                             BackArgs ba = BackArgs{}) {
    constexpr int LG = 32 / G;
    const int rs = lane & (LG - 1), gi = lane / LG;
    const int s0 = bstart[b];
    float2 X[2], Y[2], Z[2];
    RecvX2 rv;
    Comp<float> acc[2][R];
#pragma unroll
    for (int k = 0; k < 2; ++k) {
        const int li = rs + k * LG;
        const bool valid = li < nr;
        const int64_t i = s0 + r0 + (valid ? li : 0);
        const float x = loc[i], y = loc[N + i], z = loc[2 * N + i];
        X[k] = make_float2(x, x);
        Y[k] = make_float2(y, y);
        Z[k] = make_float2(z, z);
        if (SYM) {
            const float qi = valid ? q[i] : 0.f;
            rv.q[k] = make_float2(qi, qi);
        }
    }
    float *back_unit = nullptr;
    if (SYM) back_unit = ba.back + ba.base[b] + (int64_t)(r0 / P2P_UNIT) * ba.S[b];
    int boff = 0;  // owned points before the current neighbour
    const int nn = ncnt[b];
    int my_f = 0;
    float my_d[3] = {0.f, 0.f, 0.f};
    if (lane < nn) {
        my_f = nbr[b * 27 + lane];
#pragma unroll
        for (int d = 0; d < 3; ++d) my_d[d] = (float)nd[(b * 27 + lane) * 4 + d];
    }
    const int sp = lane >> 1, h = lane & 1;  // this lane's slot when staging
    for (int k = 0; k < nn; ++k) {
        const int f = __shfl_sync(0xffffffffu, my_f, k);
        const float ox = __shfl_sync(0xffffffffu, my_d[0], k);
        const float oy = __shfl_sync(0xffffffffu, my_d[1], k);
        const float oz = __shfl_sync(0xffffffffu, my_d[2], k);
        if (SYM && f < b) continue;  // uniform in the warp
        const int fs = bstart[f], fc = bcount[f];
        const bool self = (f == b);
        for (int t0 = 0; t0 < fc; t0 += 32) {
            float *a = reinterpret_cast<float *>(&sg.a[sp]);
            float *bq = reinterpret_cast<float *>(&sg.b[sp]);
            if (t0 + lane < fc) {
                const int64_t j = fs + t0 + lane;
                a[h] = -(loc[j] + ox);
                a[2 + h] = -(loc[N + j] + oy);
                bq[h] = -(loc[2 * N + j] + oz);
                bq[2 + h] = HQ ? q[j] : 0.f;
                if (HW) {
                    float *c = reinterpret_cast<float *>(&sg.c[sp]);
                    float *dd = reinterpret_cast<float *>(&sg.d[sp]);
                    c[h] = nrm[j];
                    c[2 + h] = nrm[N + j];
                    dd[h] = nrm[2 * N + j];
                    dd[2 + h] = w[j];
                }
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    if (HQ) sg.q[r - 1][lane] = q[r * N + j];
                    if (HW) sg.w[r - 1][lane] = w[r * N + j];
                }
            } else {  // zero strength, 1e4 leaf widths away
                a[h] = -1e4f;
                a[2 + h] = -1e4f;
                bq[h] = -1e4f;
                bq[2 + h] = 0.f;
                if (HW) {
                    float *c = reinterpret_cast<float *>(&sg.c[sp]);
                    float *dd = reinterpret_cast<float *>(&sg.d[sp]);
                    c[h] = 0.f;
                    c[2 + h] = 0.f;
                    dd[h] = 0.f;
                    dd[2 + h] = 0.f;
                }
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    if (HQ) sg.q[r - 1][lane] = 0.f;
                    if (HW) sg.w[r - 1][lane] = 0.f;
                }
            }
            __syncwarp();
            const int ns = min(32, fc - t0);
            if (self) p2p_tile_x2<R, G, HQ, HW, true>(sg, ns, gi, X, Y, Z, acc);
            else if constexpr (SYM) p2p_tile_x2_sym<G, HQ, HW>(sg, ns, gi, lane, X, Y, Z, rv, acc, back_unit + boff + t0);
            else p2p_tile_x2<R, G, HQ, HW, false>(sg, ns, gi, X, Y, Z, acc);
            __syncwarp();
        }
        if (SYM && !self) boff += fc;
    }
#pragma unroll
    for (int off = LG; off < 32; off <<= 1)
#pragma unroll
        for (int k = 0; k < 2; ++k)
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const float os = __shfl_xor_sync(0xffffffffu, acc[k][r].s, off);
                const float oc = __shfl_xor_sync(0xffffffffu, acc[k][r].c, off);
                acc[k][r].add(os);
                acc[k][r].c += oc;
            }
    if (gi == 0) {
#pragma unroll
        for (int k = 0; k < 2; ++k) {
            const int li = rs + k * LG;
            if (li < nr) {
                const int64_t i = s0 + r0 + li;
#pragma unroll
                for (int r = 0; r < R; ++r) out[r * N + i] = acc[k][r].get();
            }
        }
    }
}

template <int R, bool HQ, bool HW, bool SYM>
__global__ void __launch_bounds__(P2P_WARPS * 32, SYM ? 6 : (R == 1 ? 5 : 4)) k_p2p_units_x2(
    const int2 *__restrict__ units, int64_t nunits, const int32_t *__restrict__ bstart,
    const int32_t *__restrict__ bcount, const int32_t *__restrict__ nbr, const int32_t *__restrict__ ncnt,
    const int8_t *__restrict__ nd, int64_t N, const float *__restrict__ loc, const float *__restrict__ nrm,
    const float *__restrict__ q, const float *__restrict__ w, double *__restrict__ out, BackArgs ba) {
    static_assert(!SYM || (R == 1 && !HW), "the symmetric form is single-RHS, single-layer");
    __shared__ P2PStageX2<R, HQ, HW> stage[P2P_WARPS];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * P2P_WARPS;
    for (int64_t u = (int64_t)blockIdx.x * P2P_WARPS + warp; u < nunits; u += stride) {
        const int2 un = units[u];
        const int b = un.x, r0 = un.y;
        const int nr = min(P2P_UNIT, bcount[b] - r0);  // uniform in the warp
        auto &sg = stage[warp];
        if (nr > 32) p2p_unit_gx2<R, 1, HQ, HW, SYM>(sg, lane, b, r0, nr, bstart, bcount, nbr, ncnt, nd, N, loc, nrm, q, w, out, ba);
        else if (nr > 16) p2p_unit_gx2<R, 2, HQ, HW, SYM>(sg, lane, b, r0, nr, bstart, bcount, nbr, ncnt, nd, N, loc, nrm, q, w, out, ba);
        else if (nr > 8) p2p_unit_gx2<R, 4, HQ, HW, SYM>(sg, lane, b, r0, nr, bstart, bcount, nbr, ncnt, nd, N, loc, nrm, q, w, out, ba);
        else p2p_unit_gx2<R, 8, HQ, HW, SYM>(sg, lane, b, r0, nr, bstart, bcount, nbr, ncnt, nd, N, loc, nrm, q, w, out, ba);
    }
}

// Symmetric near field, second pass: one warp per work unit (up to 64 points of leaf B, two per
// lane); every point j adds the shares that the units of B's neighbours A < B wrote for it,
// neighbour by neighbour in B's list, unit by unit, in a compensated FP32 sum (TwoSum; FP64
// arithmetic is slow on this part). Lane k first looks up neighbour k's region; shuffles
// broadcast it.
constexpr int GATHER_WARPS = 8;
__global__ void __launch_bounds__(GATHER_WARPS * 32) k_p2p_back_gather(
    const int2 *__restrict__ units, int64_t nunits, const int32_t *__restrict__ bstart,
    const int32_t *__restrict__ bcount, const int32_t *__restrict__ nbr, const int32_t *__restrict__ ncnt,
    const int32_t *__restrict__ gofs, const int32_t *__restrict__ ucnt, const int32_t *__restrict__ S,
    const int64_t *__restrict__ base, const float *__restrict__ back, double *__restrict__ out) {
    const int64_t uw = (int64_t)blockIdx.x * GATHER_WARPS + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (uw >= nunits) return;  // uniform in the warp
    const int2 un = units[uw];
    const int b = un.x, r0 = un.y;
    const int nn = ncnt[b];
    int64_t my_off = 0;
    int my_S = 0, my_n = 0;
    if (lane < nn) {
        const int g = gofs[b * 27 + lane];
        if (g >= 0) {
            const int a = nbr[b * 27 + lane];
            my_off = base[a] + g;
            my_S = S[a];
            my_n = ucnt[a];
        }
    }
    const int nr = min(P2P_UNIT, bcount[b] - r0);
    const int j0 = r0 + lane, j1 = r0 + lane + 32;
    const bool v0 = lane < nr, v1 = lane + 32 < nr;
    Comp<float> a0, a1;
    for (int k = 0; k < nn; ++k) {
        const int nk = __shfl_sync(0xffffffffu, my_n, k);
        if (nk == 0) continue;
        const int64_t off = __shfl_sync(0xffffffffu, my_off, k);
        const int sk = __shfl_sync(0xffffffffu, my_S, k);
        const float *p = back + off;
        int u = 0;
        for (; u + 2 <= nk; u += 2) {  // the loads of two units issued before their (ordered) sums
            const float *pu = p + (int64_t)u * sk, *pv = pu + sk;
            const float x0 = v0 ? pu[j0] : 0.f, x1 = v1 ? pu[j1] : 0.f;
            const float y0 = v0 ? pv[j0] : 0.f, y1 = v1 ? pv[j1] : 0.f;
            a0.add(x0);
            a1.add(x1);
            a0.add(y0);
            a1.add(y1);
        }
        for (; u < nk; ++u) {
            const float *pu = p + (int64_t)u * sk;
            a0.add(v0 ? pu[j0] : 0.f);
            a1.add(v1 ? pu[j1] : 0.f);
        }
    }
    const int64_t i0 = bstart[b];
    if (v0) out[i0 + j0] += a0.get();
    if (v1) out[i0 + j1] += a1.get();
}

// Each warp takes the units u = blockIdx.x * P2P_WARPS + warp, then every gridDim.x * P2P_WARPS
// further: one unit per warp when the grid covers all units, or a persistent grid of a fixed
// number of blocks per SM (leaving room on every SM for the far-field kernels that run
// concurrently on the other stream). Every unit writes its own receivers, so the result does
// not depend on the grid.
template <class T, int R, bool HQ, bool HW>
__global__ void __launch_bounds__(P2P_WARPS * 32) k_p2p_units(
    const int2 *__restrict__ units, int64_t nunits, const int32_t *__restrict__ bstart,
    const int32_t *__restrict__ bcount, const int32_t *__restrict__ nbr, const int32_t *__restrict__ ncnt,
    const int8_t *__restrict__ nd, int64_t N, const T *__restrict__ loc, const T *__restrict__ nrm,
    const T *__restrict__ q, const T *__restrict__ w, double *__restrict__ out) {
    __shared__ P2PStage<T, R, HQ, HW> stage[P2P_WARPS];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * P2P_WARPS;
    // the loop bound is uniform in the warp; only warp-level barriers follow
    for (int64_t u = (int64_t)blockIdx.x * P2P_WARPS + warp; u < nunits; u += stride)
        p2p_unit<T, R, HQ, HW>(stage[warp], lane, units[u], bstart, bcount, nbr, ncnt, nd, N, loc, nrm, q, w, out);
}

template <int R>
struct DirArgs {
    double f[R], g[R];
    const double *xL[R];
    const double *xM[R];
    double *out[R];
};

// Direct sum in FP64 (caller's vertex order).
template <int R>
__global__ void __launch_bounds__(P2P_THREADS) k_direct64(int64_t N, const double *__restrict__ xyz, const double *__restrict__ s,
                                                          const double *__restrict__ nrm, DirArgs<R> a) {
    __shared__ double sx[P2P_THREADS], sy[P2P_THREADS], sz[P2P_THREADS];
    __shared__ double snx[P2P_THREADS], sny[P2P_THREADS], snz[P2P_THREADS];
    __shared__ double sq[R][P2P_THREADS], sw[R][P2P_THREADS];
    const int64_t i = blockIdx.x * (int64_t)P2P_THREADS + threadIdx.x;
    const bool vr = i < N;
    const int64_t ii = vr ? i : 0;
    const double xi = xyz[ii], yi = xyz[N + ii], zi = xyz[2 * N + ii];
    double acc[R];
#pragma unroll
    for (int r = 0; r < R; ++r) acc[r] = 0.0;
    for (int64_t t0 = 0; t0 < N; t0 += P2P_THREADS) {
        __syncthreads();
        int64_t j = t0 + threadIdx.x;
        if (j < N) {
            sx[threadIdx.x] = xyz[j];
            sy[threadIdx.x] = xyz[N + j];
            sz[threadIdx.x] = xyz[2 * N + j];
            snx[threadIdx.x] = nrm[j];
            sny[threadIdx.x] = nrm[N + j];
            snz[threadIdx.x] = nrm[2 * N + j];
            double sj = s[j] * kInv4Pi;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                sq[r][threadIdx.x] = a.f[r] != 0.0 ? a.f[r] * sj * a.xL[r][j] : 0.0;
                sw[r][threadIdx.x] = a.g[r] != 0.0 ? a.g[r] * sj * a.xM[r][j] : 0.0;
            }
        }
        __syncthreads();
        int ns = (int)((N - t0) < P2P_THREADS ? (N - t0) : P2P_THREADS);
        if (vr) {
            for (int sI = 0; sI < ns; ++sI) {
                double dx = xi - sx[sI], dy = yi - sy[sI], dz = zi - sz[sI];
                double r2 = dx * dx + dy * dy + dz * dz;
                double rinv = (t0 + sI == i) ? 0.0 : rsqrt(r2);
                double rinv3 = rinv * rinv * rinv;
                double nd3 = (snx[sI] * dx + sny[sI] * dy + snz[sI] * dz) * rinv3;
#pragma unroll
                for (int r = 0; r < R; ++r) acc[r] += sq[r][sI] * rinv + sw[r][sI] * nd3;
            }
        }
    }
    if (vr) {
#pragma unroll
        for (int r = 0; r < R; ++r) a.out[r][i] = acc[r];
    }
}

// Direct sum in FP32 with hi + lo coordinates and tile-compensated accumulation.
template <int R>
__global__ void __launch_bounds__(P2P_THREADS) k_direct32(int64_t N, const float *__restrict__ hi, const float *__restrict__ lo,
                                                          const double *__restrict__ s, const double *__restrict__ nrm,
                                                          DirArgs<R> a) {
    __shared__ float sxh[P2P_THREADS], syh[P2P_THREADS], szh[P2P_THREADS];
    __shared__ float sxl[P2P_THREADS], syl[P2P_THREADS], szl[P2P_THREADS];
    __shared__ float snx[P2P_THREADS], sny[P2P_THREADS], snz[P2P_THREADS];
    __shared__ float sq[R][P2P_THREADS], sw[R][P2P_THREADS];
    const int64_t i = blockIdx.x * (int64_t)P2P_THREADS + threadIdx.x;
    const bool vr = i < N;
    const int64_t ii = vr ? i : 0;
    const float xh = hi[ii], yh = hi[N + ii], zh = hi[2 * N + ii];
    const float xl = lo[ii], yl = lo[N + ii], zl = lo[2 * N + ii];
    Comp<float> acc[R];
    for (int64_t t0 = 0; t0 < N; t0 += P2P_THREADS) {
        __syncthreads();
        int64_t j = t0 + threadIdx.x;
        if (j < N) {
            sxh[threadIdx.x] = hi[j];
            syh[threadIdx.x] = hi[N + j];
            szh[threadIdx.x] = hi[2 * N + j];
            sxl[threadIdx.x] = lo[j];
            syl[threadIdx.x] = lo[N + j];
            szl[threadIdx.x] = lo[2 * N + j];
            snx[threadIdx.x] = (float)nrm[j];
            sny[threadIdx.x] = (float)nrm[N + j];
            snz[threadIdx.x] = (float)nrm[2 * N + j];
            double sj = s[j] * kInv4Pi;
#pragma unroll
            for (int r = 0; r < R; ++r) {
                sq[r][threadIdx.x] = a.f[r] != 0.0 ? (float)(a.f[r] * sj * a.xL[r][j]) : 0.f;
                sw[r][threadIdx.x] = a.g[r] != 0.0 ? (float)(a.g[r] * sj * a.xM[r][j]) : 0.f;
            }
        }
        __syncthreads();
        int ns = (int)((N - t0) < P2P_THREADS ? (N - t0) : P2P_THREADS);
        float part[R];
#pragma unroll
        for (int r = 0; r < R; ++r) part[r] = 0.f;
        if (vr) {
#pragma unroll 4
            for (int sI = 0; sI < ns; ++sI) {
                float dx = (xh - sxh[sI]) + (xl - sxl[sI]);
                float dy = (yh - syh[sI]) + (yl - syl[sI]);
                float dz = (zh - szh[sI]) + (zl - szl[sI]);
                float r2 = dx * dx + dy * dy + dz * dz;
                float rinv = (t0 + sI == i) ? 0.f : rsqrtf(r2);
                float rinv3 = rinv * rinv * rinv;
                float nd3 = (snx[sI] * dx + sny[sI] * dy + snz[sI] * dz) * rinv3;
#pragma unroll
                for (int r = 0; r < R; ++r) part[r] += sq[r][sI] * rinv + sw[r][sI] * nd3;
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r].add(part[r]);
    }
    if (vr) {
#pragma unroll
        for (int r = 0; r < R; ++r) a.out[r][i] = acc[r].get();
    }
}

}  // namespace

template <class T, int R, bool HQ, bool HW>
static void launch_units(Context &c, const T *q, const T *w, double *out_sorted, cudaStream_t st) {
    Tree &t = c.tree;
    const int L = t.L;
    const T *loc = sizeof(T) == 8 ? (const T *)t.loc64.p : (const T *)t.loc32.p;
    const T *nrm = sizeof(T) == 8 ? (const T *)t.nrm64.p : (const T *)t.nrm32.p;
    const int64_t nu = t.n_p2p_units;
    if (nu == 0) return;
    int64_t blocks = div_up(nu, P2P_WARPS);
    if (c.tuned_p2p_blocks > 0) blocks = std::min<int64_t>(blocks, (int64_t)c.num_sms * c.tuned_p2p_blocks);
    // With the far field running concurrently, ask for the SM configuration with the most shared
    // memory: the tensor-core M2L needs it, and an SM whose resident near-field blocks had it
    // configured for more L1 would first have to drain them. (A per-device attribute, set on
    // every launch; about a microsecond.)
    const int32_t *bst = t.bstart.p + t.base[L], *bcn = t.bcount.p + t.base[L];
    if constexpr (std::is_same<T, float>::value) {
        // FP32: the packed kernel, symmetric for one RHS (then the gather of the shares)
        constexpr bool SYM = R == 1 && !HW;
        auto kern = k_p2p_units_x2<R, HQ, HW, SYM>;
        if (c.tuned_overlap)
            BEM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                                          (int)cudaSharedmemCarveoutMaxShared));
        const BackArgs ba{SYM ? t.back.p : nullptr, t.back_S.p, t.back_base.p};
        kern<<<(unsigned)blocks, P2P_WARPS * 32, 0, st>>>(t.p2p_units.p, nu, bst, bcn, t.nbr.p, t.nbr_cnt.p, t.nbr_d.p,
                                                           c.N, loc, nrm, q, w, out_sorted, ba);
        BEM_LAUNCH_CHECK();
        if (SYM) {
            k_p2p_back_gather<<<(unsigned)div_up(nu, GATHER_WARPS), GATHER_WARPS * 32, 0, st>>>(
                t.p2p_units.p, nu, bst, bcn, t.nbr.p, t.nbr_cnt.p, t.back_gofs.p, t.p2p_ucnt.p, t.back_S.p,
                t.back_base.p, t.back.p, out_sorted);
        }
    } else {
        if (c.tuned_overlap)
            BEM_CUDA(cudaFuncSetAttribute(k_p2p_units<T, R, HQ, HW>, cudaFuncAttributePreferredSharedMemoryCarveout,
                                          (int)cudaSharedmemCarveoutMaxShared));
        k_p2p_units<T, R, HQ, HW><<<(unsigned)blocks, P2P_WARPS * 32, 0, st>>>(
            t.p2p_units.p, nu, bst, bcn, t.nbr.p, t.nbr_cnt.p, t.nbr_d.p, c.N, loc, nrm, q, w, out_sorted);
    }
    BEM_LAUNCH_CHECK();
}

template <class T, int R>
void launch_p2p_list(Context &c, const T *q, const T *w, double *near_sorted, bool hq, bool hw, cudaStream_t st) {
    if (R > 1 || (hq && hw)) launch_units<T, R, true, true>(c, q, w, near_sorted, st);
    else if (hw) launch_units<T, R, false, true>(c, q, w, near_sorted, st);
    else launch_units<T, R, true, false>(c, q, w, near_sorted, st);  // also the all-zero product
}

template void launch_p2p_list<float, 1>(Context &, const float *, const float *, double *, bool, bool,
                                         cudaStream_t);
template void launch_p2p_list<float, 4>(Context &, const float *, const float *, double *, bool, bool,
                                         cudaStream_t);
template void launch_p2p_list<double, 1>(Context &, const double *, const double *, double *, bool, bool,
                                         cudaStream_t);
template void launch_p2p_list<double, 4>(Context &, const double *, const double *, double *, bool, bool,
                                         cudaStream_t);

template <int R>
void launch_direct(Context &c, int prec, const double *f, const double *const *xL, const double *g,
                   const double *const *xM, double *const *out) {
    DirArgs<R> a{};
    for (int r = 0; r < R; ++r) {
        a.f[r] = f[r];
        a.g[r] = g[r];
        a.xL[r] = xL[r];
        a.xM[r] = xM[r];
        a.out[r] = out[r];
    }
    int nb = div_up(c.N, P2P_THREADS);
    PhaseScope ps(c, PH_DIRECT);
    if (prec == BEM_PREC_FP64)
        k_direct64<R><<<nb, P2P_THREADS, 0, c.stream>>>(c.N, c.xyz.p, c.s.p, c.nrm.p, a);
    else
        k_direct32<R><<<nb, P2P_THREADS, 0, c.stream>>>(c.N, c.dir_hi.p, c.dir_lo.p, c.s.p, c.nrm.p, a);
    BEM_LAUNCH_CHECK();
}

void launch_direct32_raw(int64_t N, const float *hi, const float *lo, const double *s, const double *nrm, double f,
                         const double *xL, double g, const double *xM, double *out, cudaStream_t st) {
    DirArgs<1> a{};
    a.f[0] = f;
    a.g[0] = g;
    a.xL[0] = xL;
    a.xM[0] = xM;
    a.out[0] = out;
    k_direct32<1><<<div_up(N, P2P_THREADS), P2P_THREADS, 0, st>>>(N, hi, lo, s, nrm, a);
    BEM_LAUNCH_CHECK();
}

template void launch_direct<1>(Context &, int, const double *, const double *const *, const double *,
                               const double *const *, double *const *);
template void launch_direct<4>(Context &, int, const double *, const double *const *, const double *,
                               const double *const *, double *const *);

}  // namespace bem
