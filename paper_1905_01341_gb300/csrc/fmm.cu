// Far field of the fast multipole method (Section 3.7): multipole and local expansions in
// solid harmonics of degree n = 0..p-1 (p^2 real coefficients), P2M for monopoles and
// dipoles, M2M, M2L, L2L and L2P, and the orchestration of one multi-RHS product of
// Eq. (3.27) with the near field of p2p.cu.
//
// Conventions (derived here, checked against direct sums in the tests):
//   R_n^m(r) = r^n P_n^m(cos t) e^{i m f} / (n+m)!,  I_n^m(r) = (n-m)! P_n^m(cos t) e^{i m f} / r^{n+1},
//   P_n^m with the Condon-Shortley phase, R_n^{-m} = (-1)^m conj(R_n^m), same for I. Then
//   1/|x - y| = sum_{n,m} conj(R_n^m(y)) I_n^m(x) (|y| < |x|),
//   R_n^m(a + b) = sum_{k,l} R_k^l(a) R_{n-k}^{m-l}(b),
//   d.grad R_n^m = d_z R_{n-1}^m - (d_x + i d_y)/2 R_{n-1}^{m-1} + (d_x - i d_y)/2 R_{n-1}^{m+1}.
// Expansions are normalised by the box size h of their level, so the translation matrices
// do not depend on the level: a box's field is (1/h) sum M_n^m I_n^m((x-c)/h) and its local
// expansion (1/h) sum L_n^m R_n^m((x-c)/h). Coefficients with m >= 0 are stored as reals:
// index n^2 for m = 0, n^2 + 2m - 1 (real part) and n^2 + 2m (imaginary part) for m > 0.
#include "internal.h"

#include <algorithm>
#include <cmath>

namespace bem {
namespace {

constexpr double kInv4Pi = 0.0795774715459476678844418816862571810;  // 1/(4 pi)

struct cplx {
    double re, im;
};
__device__ __forceinline__ int tri_idx(int n, int m) { return n * (n + 1) / 2 + m; }

// Harmonic of order m (any sign) from a table of m >= 0 values.
__device__ __forceinline__ cplx harm_get(const double *re, const double *im, int nmax, int n, int m) {
    if (n < 0 || n >= nmax) return {0.0, 0.0};
    int am = m < 0 ? -m : m;
    if (am > n) return {0.0, 0.0};
    double a = re[tri_idx(n, am)], b = im[tri_idx(n, am)];
    if (m >= 0) return {a, b};
    double sg = (am & 1) ? -1.0 : 1.0;
    return {sg * a, -sg * b};
}

__device__ void regular_table(double x, double y, double z, int nmax, double *re, double *im) {
    double r2 = x * x + y * y + z * z;
    double mr = 1.0, mi = 0.0;  // R_m^m
    for (int m = 0; m < nmax; ++m) {
        if (m > 0) {
            // R_m^m = -(x + i y)/(2m) R_{m-1}^{m-1}
            double f = -0.5 / m;
            double nr = f * (x * mr - y * mi), ni = f * (x * mi + y * mr);
            mr = nr;
            mi = ni;
        }
        re[tri_idx(m, m)] = mr;
        im[tri_idx(m, m)] = mi;
        if (m + 1 < nmax) {
            re[tri_idx(m + 1, m)] = z * mr;
            im[tri_idx(m + 1, m)] = z * mi;
        }
        for (int n = m + 2; n < nmax; ++n) {
            double d = 1.0 / ((double)(n + m) * (double)(n - m));
            re[tri_idx(n, m)] = ((2 * n - 1) * z * re[tri_idx(n - 1, m)] - r2 * re[tri_idx(n - 2, m)]) * d;
            im[tri_idx(n, m)] = ((2 * n - 1) * z * im[tri_idx(n - 1, m)] - r2 * im[tri_idx(n - 2, m)]) * d;
        }
    }
}

__device__ void irregular_table(double x, double y, double z, int nmax, double *re, double *im) {
    double r2 = x * x + y * y + z * z;
    double ir2 = 1.0 / r2;
    double mr = 1.0 / sqrt(r2), mi = 0.0;  // I_m^m
    for (int m = 0; m < nmax; ++m) {
        if (m > 0) {
            // I_m^m = -(2m-1)(x + i y)/r^2 I_{m-1}^{m-1}
            double f = -(2.0 * m - 1.0) * ir2;
            double nr = f * (x * mr - y * mi), ni = f * (x * mi + y * mr);
            mr = nr;
            mi = ni;
        }
        re[tri_idx(m, m)] = mr;
        im[tri_idx(m, m)] = mi;
        if (m + 1 < nmax) {
            re[tri_idx(m + 1, m)] = (2 * m + 1) * z * ir2 * mr;
            im[tri_idx(m + 1, m)] = (2 * m + 1) * z * ir2 * mi;
        }
        for (int n = m + 2; n < nmax; ++n) {
            double a = (2.0 * n - 1.0) * z * ir2, b = (double)(n + m - 1) * (double)(n - m - 1) * ir2;
            re[tri_idx(n, m)] = a * re[tri_idx(n - 1, m)] - b * re[tri_idx(n - 2, m)];
            im[tri_idx(n, m)] = a * im[tri_idx(n - 1, m)] - b * im[tri_idx(n - 2, m)];
        }
    }
}

__device__ __forceinline__ void decode(int ri, int &n, int &m, int &part) {
    n = (int)sqrtf((float)ri);
    while (n * n > ri) --n;
    while ((n + 1) * (n + 1) <= ri) ++n;
    int r = ri - n * n;
    if (r == 0) {
        m = 0;
        part = 0;
    } else if (r & 1) {
        m = (r + 1) / 2;
        part = 0;
    } else {
        m = r / 2;
        part = 1;
    }
}

constexpr int kOpM2L = 0, kOpM2M = 1, kOpL2L = 2;

__device__ cplx op_kernel(int kind, const double *hre, const double *him, int nmax, int n, int m, int k, int l) {
    if (kind == kOpM2L) {
        cplx v = harm_get(hre, him, nmax, n + k, l - m);
        double sg = ((n + m) & 1) ? -1.0 : 1.0;
        return {sg * v.re, sg * v.im};
    } else if (kind == kOpM2M) {
        if (k > n) return {0.0, 0.0};
        cplx v = harm_get(hre, him, nmax, n - k, m - l);
        double s = ldexp(1.0, -k);
        return {s * v.re, -s * v.im};
    } else {
        if (k < n) return {0.0, 0.0};
        cplx v = harm_get(hre, him, nmax, k - n, l - m);
        double s = ldexp(1.0, -n - 1);
        return {s * v.re, s * v.im};
    }
}

// One block per matrix. M2L: offset class -> D = target centre - source centre in units of
// the box (the class enumerates source - target offsets lexicographically). M2M/L2L: child
// octant o -> t = child centre - parent centre in units of the parent box.
__global__ void k_build_ops(int kind, int p, double *__restrict__ out64, float *__restrict__ out32) {
    extern __shared__ double sh[];
    const int P = p * p;
    const int nmax = (kind == kOpM2L) ? 2 * p : p;
    const int ntri = nmax * (nmax + 1) / 2;
    double *hre = sh, *him = sh + ntri;
    if (threadIdx.x == 0) {
        double v[3];
        if (kind == kOpM2L) {
            int c = 0, want = blockIdx.x;
            for (int x = -3; x <= 3; ++x)
                for (int y = -3; y <= 3; ++y)
                    for (int z = -3; z <= 3; ++z) {
                        bool near = (x >= -1 && x <= 1 && y >= -1 && y <= 1 && z >= -1 && z <= 1);
                        if (near) continue;
                        if (c == want) {
                            v[0] = -x;
                            v[1] = -y;
                            v[2] = -z;
                        }
                        ++c;
                    }
            irregular_table(v[0], v[1], v[2], nmax, hre, him);
        } else {
            int o = blockIdx.x;
            v[0] = (((o >> 2) & 1) - 0.5) * 0.5;
            v[1] = (((o >> 1) & 1) - 0.5) * 0.5;
            v[2] = ((o & 1) - 0.5) * 0.5;
            regular_table(v[0], v[1], v[2], nmax, hre, him);
        }
    }
    __syncthreads();
    size_t mbase = (size_t)blockIdx.x * P * P;
    for (int e = threadIdx.x; e < P * P; e += blockDim.x) {
        int ro = e / P, ri = e % P;
        int n, m, po, k, l, pi;
        decode(ro, n, m, po);
        decode(ri, k, l, pi);
        double val;
        if (l == 0) {
            cplx c = op_kernel(kind, hre, him, nmax, n, m, k, 0);
            val = (pi != 0) ? 0.0 : (po == 0 ? c.re : c.im);
        } else {
            cplx kp = op_kernel(kind, hre, him, nmax, n, m, k, l);
            cplx km = op_kernel(kind, hre, him, nmax, n, m, k, -l);
            double sg = (l & 1) ? -1.0 : 1.0;
            cplx A = {kp.re + sg * km.re, kp.im + sg * km.im};
            cplx B = {kp.re - sg * km.re, kp.im - sg * km.im};
            if (po == 0) val = (pi == 0) ? A.re : -B.im;
            else val = (pi == 0) ? A.im : B.re;
        }
        out64[mbase + e] = val;
        out32[mbase + e] = (float)val;
    }
}

// ------------------------------------------------------------------------------ strengths
template <int R>
struct RhsArgs {
    double f[R], g[R];
    const double *xL[R];
    const double *xM[R];
    double *out[R];
};

// Monopole q = f s X_L / (4 pi) and dipole moment w n with w = g s X_M / (4 pi) / h_leaf
// (leaf-box units), gathered into Morton order.
template <class T, int R>
__global__ void k_strengths(int64_t N, const int32_t *__restrict__ perm, const double *__restrict__ s,
                            RhsArgs<R> a, const double *__restrict__ ih, T *__restrict__ q, T *__restrict__ w) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= N) return;
    int j = perm[k];
    double sk = s[k] * kInv4Pi;
    const double inv_h = ih[k];
#pragma unroll
    for (int r = 0; r < R; ++r) {
        double qq = a.f[r] != 0.0 ? a.f[r] * sk * a.xL[r][j] : 0.0;
        double ww = a.g[r] != 0.0 ? a.g[r] * sk * a.xM[r][j] * inv_h : 0.0;
        q[r * N + k] = (T)qq;
        w[r * N + k] = (T)ww;
    }
}

// ------------------------------------------------------------------------------ P2M
// One block per leaf. Points are taken 32 at a time: their regular harmonics R_n^m (m >= 0)
// are built column by column (the recurrence in n for each m) into shared memory, then each
// thread owns one complex coefficient (n, m) and accumulates
//   M_n^m += q conj(R_n^m) + w conj(n . grad R_n^m),
//   n . grad R_n^m = n_z R_{n-1}^m - (n_x + i n_y)/2 R_{n-1}^{m-1} + (n_x - i n_y)/2 R_{n-1}^{m+1},
// over the points, for the real and imaginary part together.
constexpr int P2M_PC = 32;  // points per chunk

template <class T>
struct Vec2 {
    using type = float2;
};
template <>
struct Vec2<double> {
    using type = double2;
};

template <class T, int R, bool HW>
__global__ void __launch_bounds__(256) k_p2m(int p, int nleaf, const int32_t *__restrict__ bstart,
                                             const int32_t *__restrict__ bcount, int64_t N,
                                             const T *__restrict__ loc, const T *__restrict__ nrm,
                                             const T *__restrict__ q, const T *__restrict__ w,
                                             T *__restrict__ mp) {
    using T2 = typename Vec2<T>::type;
    extern __shared__ __align__(16) unsigned char smraw[];
    const int P = p * p;
    const int ntri = p * (p + 1) / 2;
    T2 *Rt = reinterpret_cast<T2 *>(smraw);          // [PC][ntri]
    T *pn = reinterpret_cast<T *>(Rt + P2M_PC * ntri);  // [PC][3]
    T *pq = pn + P2M_PC * 3;                            // [PC][R]
    T *pw = pq + P2M_PC * R;                            // [PC][R]
    T *tk = pw + P2M_PC * R;                            // [p]: -1 / (2k)
    T *tnm = tk + p;                                    // [ntri]: 1 / ((n + m)(n - m)), n >= m + 2
    for (int e = threadIdx.x; e < p; e += blockDim.x) tk[e] = e > 0 ? (T)(-0.5) / (T)e : (T)0;
    for (int e = threadIdx.x; e < ntri; e += blockDim.x) {
        int n = 0;
        while ((n + 1) * (n + 2) / 2 <= e) ++n;
        const int m = e - n * (n + 1) / 2;
        tnm[e] = n >= m + 2 ? (T)1 / ((T)(n + m) * (T)(n - m)) : (T)0;
    }
    const int b = blockIdx.x;
    const int s0 = bstart[b], cnt = bcount[b];
    constexpr int MAXC = 2;  // complex coefficients per thread (ntri <= 2 * blockDim)
    int cn[MAXC], cm[MAXC];
    T are[MAXC][R], aim[MAXC][R];
#pragma unroll
    for (int o = 0; o < MAXC; ++o) {
        int c = threadIdx.x + o * blockDim.x;
        int n = 0;
        while ((n + 1) * (n + 2) / 2 <= c) ++n;
        cn[o] = (c < ntri) ? n : -1;
        cm[o] = c - n * (n + 1) / 2;
#pragma unroll
        for (int r = 0; r < R; ++r) are[o][r] = aim[o][r] = (T)0;
    }
    for (int c0 = 0; c0 < cnt; c0 += P2M_PC) {
        const int pc = min(P2M_PC, cnt - c0);
        __syncthreads();
        if (HW)
            for (int e = threadIdx.x; e < pc * 3; e += blockDim.x) {
                int jj = e / 3, d = e % 3;
                pn[jj * 3 + d] = nrm[d * N + s0 + c0 + jj];
            }
        for (int e = threadIdx.x; e < pc * R; e += blockDim.x) {
            int jj = e / R, r = e % R;
            pq[jj * R + r] = q[r * N + s0 + c0 + jj];
            pw[jj * R + r] = HW ? w[r * N + s0 + c0 + jj] : (T)0;
        }
        // each task: one order m for four points (independent recurrences in flight). The point
        // groups vary fastest, so a warp's lanes share a few neighbouring orders and run nearly
        // the same trip counts through the m loop and the n loop (orders mixed across the lanes
        // made every warp run the longest of both loops)
        const int ngroups = (pc + 3) / 4;
        for (int task = threadIdx.x; task < ngroups * p; task += blockDim.x) {
            const int g = task % ngroups, m = task / ngroups;
            T x[4], y[4], z[4], r2[4], mr[4], mi[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const int jj = min(g * 4 + u, pc - 1);
                const int64_t i = s0 + c0 + jj;
                x[u] = loc[i];
                y[u] = loc[N + i];
                z[u] = loc[2 * N + i];
                r2[u] = x[u] * x[u] + y[u] * y[u] + z[u] * z[u];
                mr[u] = 1;
                mi[u] = 0;
            }
            for (int k = 1; k <= m; ++k) {
                const T f = tk[k];  // -1 / (2k)
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const T nr = f * (x[u] * mr[u] - y[u] * mi[u]), ni = f * (x[u] * mi[u] + y[u] * mr[u]);
                    mr[u] = nr;
                    mi[u] = ni;
                }
            }
            T p2r[4], p2i[4], p1r[4], p1i[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                T2 *col = Rt + (g * 4 + u) * ntri;
                const bool ok = g * 4 + u < pc;
                if (ok) col[tri_idx(m, m)] = T2{mr[u], mi[u]};
                p2r[u] = mr[u];
                p2i[u] = mi[u];
                p1r[u] = z[u] * mr[u];
                p1i[u] = z[u] * mi[u];
                if (ok && m + 1 < p) col[tri_idx(m + 1, m)] = T2{p1r[u], p1i[u]};
            }
            for (int n = m + 2; n < p; ++n) {
                const int idx = tri_idx(n, m);
                const T d = tnm[idx];  // 1 / ((n + m)(n - m))
                const T c2 = (T)(2 * n - 1);
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    const T cr = (c2 * z[u] * p1r[u] - r2[u] * p2r[u]) * d;
                    const T ci = (c2 * z[u] * p1i[u] - r2[u] * p2i[u]) * d;
                    if (g * 4 + u < pc) Rt[(g * 4 + u) * ntri + idx] = T2{cr, ci};
                    p2r[u] = p1r[u];
                    p2i[u] = p1i[u];
                    p1r[u] = cr;
                    p1i[u] = ci;
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int o = 0; o < MAXC; ++o) {
            const int n = cn[o], m = cm[o];
            if (n < 0) continue;
            const int iA = tri_idx(n, m);
            const int iB = (n >= 1 && m <= n - 1) ? tri_idx(n - 1, m) : -1;
            const int iL = (n >= 1 && m >= 1) ? tri_idx(n - 1, m - 1) : ((n >= 2) ? tri_idx(n - 1, 1) : -1);
            const int iU = (n >= 1 && m + 1 <= n - 1) ? tri_idx(n - 1, m + 1) : -1;
            const bool neg1 = (m == 0);  // R^{-1} = -conj(R^1)
            for (int jj = 0; jj < pc; ++jj) {
                const T2 *col = Rt + jj * ntri;
                const T2 A = col[iA];
                T gr = 0, gi = 0;
                if (HW && n >= 1) {
                    const T nx = pn[jj * 3], ny = pn[jj * 3 + 1], nz = pn[jj * 3 + 2];
                    T2 Bm = iB >= 0 ? col[iB] : T2{0, 0};
                    T2 Bl = iL >= 0 ? col[iL] : T2{0, 0};
                    if (neg1) Bl = T2{-Bl.x, Bl.y};
                    T2 Bu = iU >= 0 ? col[iU] : T2{0, 0};
                    gr = nz * Bm.x - (T)0.5 * (nx * Bl.x - ny * Bl.y) + (T)0.5 * (nx * Bu.x + ny * Bu.y);
                    gi = nz * Bm.y - (T)0.5 * (nx * Bl.y + ny * Bl.x) + (T)0.5 * (nx * Bu.y - ny * Bu.x);
                }
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const T qq = pq[jj * R + r];
                    if (HW) {
                        const T ww = pw[jj * R + r];
                        are[o][r] += qq * A.x + ww * gr;
                        aim[o][r] -= qq * A.y + ww * gi;
                    } else {
                        are[o][r] += qq * A.x;
                        aim[o][r] -= qq * A.y;
                    }
                }
            }
        }
    }
#pragma unroll
    for (int o = 0; o < MAXC; ++o) {
        const int n = cn[o], m = cm[o];
        if (n < 0) continue;
#pragma unroll
        for (int r = 0; r < R; ++r) {
            T *dst = mp + ((size_t)b * R + r) * P;
            if (m == 0) {
                dst[n * n] = are[o][r];
            } else {
                dst[n * n + 2 * m - 1] = are[o][r];
                dst[n * n + 2 * m] = aim[o][r];
            }
        }
    }
}

// FP32 single-RHS, single-layer P2M (every GMRES product) in packed two-wide arithmetic
// (add/mul/fma .f32x2). The same two phases as k_p2m, with the harmonics of a chunk stored as
// planes re[ntri][P2MX_RS], im[ntri][P2MX_RS] (point index fastest, rows padded against bank
// conflicts): a recurrence task (order m, four points) runs as two packed pairs of points and
// stores each pair with one 8-byte store; a coefficient's thread sums q x R over the chunk's
// points two at a time (q of the points past the chunk's end is zero, their harmonics finite).
constexpr int P2MX_RS = P2M_PC + 2;
__global__ void __launch_bounds__(128) k_p2m_x2(int p, int nleaf, const int32_t *__restrict__ bstart,
                                                const int32_t *__restrict__ bcount, int64_t N,
                                                const float *__restrict__ loc, const float *__restrict__ q,
                                                float *__restrict__ mp) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int P = p * p;
    const int ntri = p * (p + 1) / 2;
    float *re = reinterpret_cast<float *>(smraw);  // [ntri][P2MX_RS]
    float *im = re + ntri * P2MX_RS;               // [ntri][P2MX_RS]
    float *pq = im + ntri * P2MX_RS;               // [P2M_PC]
    float2 *tk = reinterpret_cast<float2 *>(pq + P2M_PC);  // [p]: -1 / (2k)
    float2 *c2t = tk + p;                                  // [p]: 2n - 1
    float2 *tnm = c2t + p;                                 // [ntri]: 1 / ((n + m)(n - m)), n >= m + 2
    for (int e = threadIdx.x; e < p; e += blockDim.x) {
        const float v = e > 0 ? -0.5f / (float)e : 0.f, c = (float)(2 * e - 1);
        tk[e] = make_float2(v, v);
        c2t[e] = make_float2(c, c);
    }
    for (int e = threadIdx.x; e < ntri; e += blockDim.x) {
        int n = 0;
        while ((n + 1) * (n + 2) / 2 <= e) ++n;
        const int m = e - n * (n + 1) / 2;
        const float v = n >= m + 2 ? 1.f / ((float)(n + m) * (float)(n - m)) : 0.f;
        tnm[e] = make_float2(v, v);
    }
    const int b = blockIdx.x;
    const int s0 = bstart[b], cnt = bcount[b];
    constexpr int MAXC = 2;  // complex coefficients per thread (ntri <= 2 * blockDim)
    int cn[MAXC], cm[MAXC];
    float2 accr[MAXC], acci[MAXC];
#pragma unroll
    for (int o = 0; o < MAXC; ++o) {
        const int c = threadIdx.x + o * blockDim.x;
        int n = 0;
        while ((n + 1) * (n + 2) / 2 <= c) ++n;
        cn[o] = (c < ntri) ? n : -1;
        cm[o] = c - n * (n + 1) / 2;
        accr[o] = acci[o] = make_float2(0.f, 0.f);
    }
    for (int c0 = 0; c0 < cnt; c0 += P2M_PC) {
        const int pc = min(P2M_PC, cnt - c0);
        __syncthreads();
        for (int jj = threadIdx.x; jj < P2M_PC; jj += blockDim.x) pq[jj] = jj < pc ? q[s0 + c0 + jj] : 0.f;
        // recurrence tasks: (order m, four points), the point groups fastest
        constexpr int NG = P2M_PC / 4;
        for (int task = threadIdx.x; task < NG * p; task += blockDim.x) {
            const int g = task % NG, m = task / NG;
            float2 X[2], Y[2], Z[2], NR2[2], MR[2], MI[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int64_t ia = s0 + c0 + min(g * 4 + 2 * h, pc - 1), ib = s0 + c0 + min(g * 4 + 2 * h + 1, pc - 1);
                X[h] = make_float2(loc[ia], loc[ib]);
                Y[h] = make_float2(loc[N + ia], loc[N + ib]);
                Z[h] = make_float2(loc[2 * N + ia], loc[2 * N + ib]);
                const float2 r2 = __ffma2_rn(Z[h], Z[h], __ffma2_rn(Y[h], Y[h], __fmul2_rn(X[h], X[h])));
                NR2[h] = make_float2(-r2.x, -r2.y);
                MR[h] = make_float2(1.f, 1.f);
                MI[h] = make_float2(0.f, 0.f);
            }
            for (int k = 1; k <= m; ++k) {
                const float2 F = tk[k];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float2 a = __ffma2_rn(X[h], MR[h], __fmul2_rn(make_float2(-Y[h].x, -Y[h].y), MI[h]));
                    const float2 bb = __ffma2_rn(X[h], MI[h], __fmul2_rn(Y[h], MR[h]));
                    MR[h] = __fmul2_rn(F, a);
                    MI[h] = __fmul2_rn(F, bb);
                }
            }
            float2 P2R[2], P2I[2], P1R[2], P1I[2];
            const int rmm = tri_idx(m, m) * P2MX_RS + g * 4, rm1 = tri_idx(m + 1, m) * P2MX_RS + g * 4;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                *reinterpret_cast<float2 *>(re + rmm + 2 * h) = MR[h];
                *reinterpret_cast<float2 *>(im + rmm + 2 * h) = MI[h];
                P2R[h] = MR[h];
                P2I[h] = MI[h];
                P1R[h] = __fmul2_rn(Z[h], MR[h]);
                P1I[h] = __fmul2_rn(Z[h], MI[h]);
                if (m + 1 < p) {
                    *reinterpret_cast<float2 *>(re + rm1 + 2 * h) = P1R[h];
                    *reinterpret_cast<float2 *>(im + rm1 + 2 * h) = P1I[h];
                }
            }
            for (int n = m + 2; n < p; ++n) {
                const int idx = tri_idx(n, m);
                const float2 D = tnm[idx], C2 = c2t[n];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const float2 C2Z = __fmul2_rn(C2, Z[h]);
                    const float2 CR = __fmul2_rn(__ffma2_rn(C2Z, P1R[h], __fmul2_rn(NR2[h], P2R[h])), D);
                    const float2 CI = __fmul2_rn(__ffma2_rn(C2Z, P1I[h], __fmul2_rn(NR2[h], P2I[h])), D);
                    *reinterpret_cast<float2 *>(re + idx * P2MX_RS + g * 4 + 2 * h) = CR;
                    *reinterpret_cast<float2 *>(im + idx * P2MX_RS + g * 4 + 2 * h) = CI;
                    P2R[h] = P1R[h];
                    P2I[h] = P1I[h];
                    P1R[h] = CR;
                    P1I[h] = CI;
                }
            }
        }
        __syncthreads();
#pragma unroll
        for (int o = 0; o < MAXC; ++o) {
            if (cn[o] < 0) continue;
            const int row = tri_idx(cn[o], cm[o]) * P2MX_RS;
#pragma unroll 4
            for (int jj = 0; jj < P2M_PC; jj += 2) {
                const float2 Q = *reinterpret_cast<const float2 *>(pq + jj);
                accr[o] = __ffma2_rn(Q, *reinterpret_cast<const float2 *>(re + row + jj), accr[o]);
                acci[o] = __ffma2_rn(Q, *reinterpret_cast<const float2 *>(im + row + jj), acci[o]);
            }
        }
    }
#pragma unroll
    for (int o = 0; o < MAXC; ++o) {
        const int n = cn[o], m = cm[o];
        if (n < 0) continue;
        float *dst = mp + (size_t)b * P;
        if (m == 0) {
            dst[n * n] = accr[o].x + accr[o].y;
        } else {
            dst[n * n + 2 * m - 1] = accr[o].x + accr[o].y;
            dst[n * n + 2 * m] = -(acci[o].x + acci[o].y);
        }
    }
}

// ------------------------------------------------------------------------------ translations
// Class-grouped product: for every pair (src, tgt) of a chunk, Y[tgt] += T_cls X[src], as a
// tiled GEMM (128 output rows x 128 columns per block in FP32, 64 x 64 in FP64; a column is one
// pair and one RHS).
constexpr int XT_K = 16, XT_THREADS = 256;

// MODE kStorePair: Y[pair] = T X[src] (one slot per pair, summed later in a fixed order).
// MODE kAddTarget: Y[tgt] += T X[src]; only for launches whose targets are all distinct.
constexpr int kStorePair = 0, kAddTarget = 1;

// N consecutive elements (16 bytes) from shared memory
template <int N>
__device__ __forceinline__ void vec_load(const float *p, float *v) {
    static_assert(N == 4, "16-byte loads");
    const float4 t = *reinterpret_cast<const float4 *>(p);
    v[0] = t.x;
    v[1] = t.y;
    v[2] = t.z;
    v[3] = t.w;
}
template <int N>
__device__ __forceinline__ void vec_load(const double *p, double *v) {
    static_assert(N == 2, "16-byte loads");
    const double2 t = *reinterpret_cast<const double2 *>(p);
    v[0] = t.x;
    v[1] = t.y;
}

// outputs per thread and block: 8 x 8 per thread in FP32 (a 128 x 128 tile: 16 FMAs per shared
// load, and each operator tile serves 128 (pair, rhs) columns), 4 x 4 in FP64 (64 x 64, which
// keeps two blocks of three stages per SM)
template <class T>
__host__ __device__ constexpr int xt_rt() { return sizeof(T) == 4 ? 8 : 4; }
template <class T>
__host__ __device__ constexpr int xt_rows() { return 16 * xt_rt<T>(); }
template <class T>
__host__ __device__ constexpr int xt_cols() { return 16 * xt_rt<T>(); }
// row pitches of the shared-memory stages: multiples of 16 bytes
template <class T>
__host__ __device__ constexpr int xt_apitch() { return xt_rows<T>() + 4; }
template <class T>
__host__ __device__ constexpr int xt_bpitch() { return xt_cols<T>() + 4; }
constexpr int XT_STAGES = 3;
template <class T>
constexpr size_t xt_smem() { return (size_t)XT_STAGES * XT_K * (xt_apitch<T>() + xt_bpitch<T>()) * sizeof(T); }

// one element global -> shared without a register round trip; ok = false writes zero
template <class T>
__device__ __forceinline__ void cp_async_elem(T *dst, const T *src, bool ok) {
    const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(d), "l"(src), "n"((int)sizeof(T)),
                 "r"(ok ? (int)sizeof(T) : 0)
                 : "memory");
}

template <class T, int R, int MODE>
__global__ void __launch_bounds__(XT_THREADS, 2) k_xlat(const T *__restrict__ mats, int P, const XChunk *__restrict__ chunks,
                                                     const int32_t *__restrict__ srcs, const int32_t *__restrict__ tgts,
                                                     const T *X, T *Y,  // X and Y may be one array (M2M, L2L)
                                                     const int32_t *__restrict__ cls_K) {
    constexpr int RT = xt_rt<T>(), CT = RT, ROWS = xt_rows<T>(), COLS = xt_cols<T>();
    constexpr int AP = xt_apitch<T>(), BP = xt_bpitch<T>(), VW = 16 / (int)sizeof(T);
    // XT_STAGES shared-memory stages of one K tile each: As[st][kk][row], Bs[st][kk][col]
    extern __shared__ __align__(16) unsigned char xt_smem_raw[];
    T *As = reinterpret_cast<T *>(xt_smem_raw);
    T *Bs = As + XT_STAGES * XT_K * AP;
    __shared__ int s_src[COLS], s_tgt[COLS];
    const XChunk ch = chunks[blockIdx.x];
    const int row0 = blockIdx.y * ROWS;
    const T *A = mats + (size_t)ch.cls * P * P;
    // truncated translation of this class (M2L with per-class orders): inputs and outputs of
    // index < Kt; output rows from Kt on are written as zeros (kStorePair)
    const int Kt = cls_K ? min(P, cls_K[ch.cls]) : P;
    const int ncol = ch.count * R;
    int tid = threadIdx.x;
    for (int e = tid; e < COLS; e += XT_THREADS) {
        int pr = e / R;
        if (pr < ch.count) {
            s_src[e] = srcs[ch.start + pr];
            s_tgt[e] = tgts[ch.start + pr];
        } else {
            s_src[e] = -1;
            s_tgt[e] = -1;
        }
    }
    __syncthreads();
    // a warp is an 8 x 4 grid of lanes (8 column groups, 4 row groups) and the block 2 x 4 warps;
    // thread (tx, ty) owns the columns tx*CH.. and COLS/2 + tx*CH.. and the rows ty*RH.. and
    // ROWS/2 + ty*RH.., so each 16-byte shared-memory load of a warp reads one contiguous run of
    // 128 bytes (multipoles) or 64 bytes (operator, broadcast within the warp): one wavefront
    constexpr int RH = RT / 2, CH = CT / 2;
    const int lane = tid & 31, wid = tid >> 5;
    const int tx = (wid & 1) * 8 + (lane & 7), ty = (wid >> 1) * 4 + (lane >> 3);
    auto row_of = [&](int i) { return i < RH ? ty * RH + i : ROWS / 2 + ty * RH + (i - RH); };
    auto col_of = [&](int j) { return j < CH ? tx * CH + j : COLS / 2 + tx * CH + (j - CH); };
    T acc[RT][CT];
#pragma unroll
    for (int i = 0; i < RT; ++i)
#pragma unroll
        for (int j = 0; j < CT; ++j) acc[i][j] = (T)0;
    constexpr int NA = (ROWS * XT_K) / XT_THREADS, NB = (COLS * XT_K) / XT_THREADS;
    // stage st <- the K tile at k0, copied straight from global memory (element-wise cp.async;
    // zero-filled outside the operator and past the last column); one commit group per call
    auto cpload = [&](int k0, int st) {
#pragma unroll
        for (int it = 0; it < NA; ++it) {
            const int e = tid + it * XT_THREADS;
            const int row = e / XT_K, kk = e % XT_K;
            const int gr = row0 + row, gk = k0 + kk;
            const bool ok = gr < Kt && gk < Kt;
            const T *src = A + (ok ? (size_t)gr * P + gk : 0);
            cp_async_elem(As + (st * XT_K + kk) * AP + row, src, ok);
        }
#pragma unroll
        for (int it = 0; it < NB; ++it) {
            const int e = tid + it * XT_THREADS;
            const int col = e / XT_K, kk = e % XT_K;
            const int gk = k0 + kk;
            const bool ok = col < ncol && gk < Kt;
            const T *src = X + (ok ? ((size_t)s_src[col] * R + col % R) * P + gk : 0);
            cp_async_elem(Bs + (st * XT_K + kk) * BP + col, src, ok);
        }
        asm volatile("cp.async.commit_group;" ::: "memory");
    };
    const int nk = (Kt + XT_K - 1) / XT_K;
    // three stages: tiles t + 1 and t + 2 are in flight while tile t is multiplied
    cpload(0, 0);
    if (nk > 1) cpload(XT_K, 1);
    else asm volatile("cp.async.commit_group;" ::: "memory");
    for (int t = 0; t < nk; ++t) {
        const int buf = t % XT_STAGES;
        asm volatile("cp.async.wait_group 1;" ::: "memory");  // tile t has landed (this thread's part)
        // every thread's part of tile t is visible, and the stage of tile t - 1 is no longer read
        __syncthreads();
        if (t + 2 < nk) cpload((t + 2) * XT_K, (t + 2) % XT_STAGES);
        else asm volatile("cp.async.commit_group;" ::: "memory");  // keeps one group per iteration
        if (row0 + ty * RH < Kt && tx * CH < ncol) {  // rows past Kt and empty columns skip the products
#pragma unroll
            for (int kk = 0; kk < XT_K; ++kk) {
                // two runs of consecutive rows / columns per thread, 16 bytes per load
                const T *as = As + (buf * XT_K + kk) * AP, *bs = Bs + (buf * XT_K + kk) * BP;
                T a[RT], bv[CT];
#pragma unroll
                for (int v = 0; v < RH; v += VW) {
                    vec_load<VW>(as + ty * RH + v, a + v);
                    vec_load<VW>(as + ROWS / 2 + ty * RH + v, a + RH + v);
                }
#pragma unroll
                for (int v = 0; v < CH; v += VW) {
                    vec_load<VW>(bs + tx * CH + v, bv + v);
                    vec_load<VW>(bs + COLS / 2 + tx * CH + v, bv + CH + v);
                }
#pragma unroll
                for (int i = 0; i < RT; ++i)
#pragma unroll
                    for (int j = 0; j < CT; ++j) acc[i][j] += a[i] * bv[j];
            }
        }
    }
#pragma unroll
    for (int j = 0; j < CT; ++j) {
        int col = col_of(j);
        if (col >= ncol) continue;
        int r = col % R;
        T *yb = (MODE == kStorePair) ? Y + ((size_t)(ch.start + col / R) * R + r) * P
                                     : Y + ((size_t)s_tgt[col] * R + r) * P;
#pragma unroll
        for (int i = 0; i < RT; ++i) {
            int gr = row0 + row_of(i);
            if (gr < Kt) {  // truncated rows (Kt < P) are never read
                if (MODE == kStorePair) yb[gr] = acc[i][j];
                else yb[gr] += acc[i][j];
            }
        }
    }
}

// dynamic shared memory above the 48 KB default needs an opt-in, which belongs to the current
// device: set before every launch (a host call of about a microsecond)
template <class K>
void xlat_smem_attr(K kern, size_t bytes) {
    if (bytes > 48 * 1024) BEM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
}

// Y[t] += sum of Ypair[k] over the pairs k of target t, in ascending k (fixed order,
// compensated in FP32). One thread per (target, coefficient).
// With per-class truncation (byK != nullptr: byK[k] is the truncated size of the class of pair
// by[k]) a pair's row holds only its class's first byK coefficients; the rest were never
// written and count as zeros (skipping a zero leaves a TwoSum accumulation unchanged, so the
// result is the same as summing the zeros).
template <class T, int R>
__global__ void k_reduce_pairs(int t0, const int32_t *__restrict__ off, const int32_t *__restrict__ by,
                               const T *__restrict__ Ypair, int P, T *__restrict__ Y, const int32_t *__restrict__ byK) {
    int t = t0 + blockIdx.x;
    int e = blockIdx.y * blockDim.x + threadIdx.x;
    if (e >= R * P) return;
    int a = off[t], b = off[t + 1];
    if (a == b) return;
    const int n = e % P;
    T s = 0, c = 0;
    for (int k = a; k < b; ++k) {
        if (byK && n >= byK[k]) continue;
        T v = Ypair[(size_t)by[k] * R * P + e];
        T tt = s + v;
        T bp = tt - s;
        c += (s - (tt - bp)) + (v - bp);
        s = tt;
    }
    Y[(size_t)t * R * P + e] += s + c;
}

// FP32 with R*P a multiple of 4: one 64-thread block per target, each thread four consecutive
// coefficients through 16-byte loads, two product rows in flight. Per coefficient the order and
// the arithmetic are those of k_reduce_pairs, so the results are the same bit for bit.
__device__ __forceinline__ void comp_add(float &s, float &c, float v) {
    const float tt = s + v;
    const float bp = tt - s;
    c += (s - (tt - bp)) + (v - bp);
    s = tt;
}
template <int R>
__global__ void __launch_bounds__(64) k_reduce_pairs4(int t0, const int32_t *__restrict__ off,
                                                      const int32_t *__restrict__ by, const float *__restrict__ Ypair,
                                                      int P, float *__restrict__ Y, const int32_t *__restrict__ byK) {
    const int t = t0 + blockIdx.x;
    const int a = off[t], b = off[t + 1];
    if (a == b) return;
    const int rp4 = R * P / 4;
    const float4 *Y4 = reinterpret_cast<const float4 *>(Ypair);
    for (int e = threadIdx.x; e < rp4; e += blockDim.x) {
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f, c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
        auto add = [&](const float4 v) {
            comp_add(s0, c0, v.x);
            comp_add(s1, c1, v.y);
            comp_add(s2, c2, v.z);
            comp_add(s3, c3, v.w);
        };
        if (byK) {
            // truncated classes: the four coefficients (4e .. 4e + 3) % P lie on one side of the
            // pair's class size byK[k] (a multiple of 16) together
            const int n = (4 * e) % P;
            const float4 z = make_float4(0.f, 0.f, 0.f, 0.f);
            int k = a;
            for (; k + 3 < b; k += 4) {  // four rows in flight, added in pair order
                float4 v[4];
                bool in[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) {
                    in[u] = n < byK[k + u];
                    v[u] = in[u] ? Y4[(size_t)by[k + u] * rp4 + e] : z;
                }
#pragma unroll
                for (int u = 0; u < 4; ++u)
                    if (in[u]) add(v[u]);
            }
            for (; k < b; ++k)
                if (n < byK[k]) add(Y4[(size_t)by[k] * rp4 + e]);
        } else {
            int k = a;
            for (; k + 3 < b; k += 4) {
                float4 v[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) v[u] = Y4[(size_t)by[k + u] * rp4 + e];
#pragma unroll
                for (int u = 0; u < 4; ++u) add(v[u]);
            }
            for (; k < b; ++k) add(Y4[(size_t)by[k] * rp4 + e]);
        }
        float4 *dst = reinterpret_cast<float4 *>(Y) + (size_t)t * rp4 + e;
        float4 y = *dst;
        y.x += s0 + c0;
        y.y += s1 + c1;
        y.z += s2 + c2;
        y.w += s3 + c3;
        *dst = y;
    }
}

// Y[t] += sum over the pairs of t, for the targets t0 .. t0 + ntg - 1
// byK[k] = cls_K[class of pair by[k]]: the truncated row length, in the target-major order
__global__ void k_pair_K(int64_t n, const int32_t *__restrict__ by, const uint32_t *__restrict__ pair_cls,
                         const int32_t *__restrict__ cls_K, int32_t *__restrict__ byK) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k < n) byK[k] = cls_K[pair_cls[by[k]]];
}

template <class T, int R>
void launch_reduce_pairs(int t0, int ntg, const int32_t *off, const int32_t *by, const T *Ypair, int P, T *Y,
                         cudaStream_t st, const int32_t *byK = nullptr) {
    if (ntg <= 0) return;
    if constexpr (sizeof(T) == 4) {
        if (P % 4 == 0) {
            k_reduce_pairs4<R><<<ntg, 64, 0, st>>>(t0, off, by, Ypair, P, Y, byK);
            BEM_LAUNCH_CHECK();
            return;
        }
    }
    dim3 rg((unsigned)ntg, div_up(R * P, 128));
    k_reduce_pairs<T, R><<<rg, 128, 0, st>>>(t0, off, by, Ypair, P, Y, byK);
    BEM_LAUNCH_CHECK();
}

// ------------------------------------------------------------------------------ L2P
// One warp per leaf: leaves hold about 70-150 points, and a 128-thread block left most of its
// lanes idle on the second pass over a leaf's points.
constexpr int L2P_THREADS = 32;

// TwoSum-compensated accumulation in T; for double the compensation is harmless.
template <class T>
struct CompSum {
    T s = 0, c = 0;
    __device__ __forceinline__ void add(T v) {
        T t = s + v;
        T bp = t - s;
        c += (s - (t - bp)) + (v - bp);
        s = t;
    }
    __device__ __forceinline__ T get() const { return s + c; }
};

// far_i = sum_{n,m} L_n^m R_n^m(x_i) at the leaf's points (real form: m = 0 once, m > 0 twice the
// real part). The regular harmonics come from the same recurrences as in P2M, column by column
// (fixed m, rising n), with tabulated divisors; each column is summed plainly and the columns are
// merged with compensation.
template <class T, int R>
__global__ void __launch_bounds__(L2P_THREADS) k_l2p(int p, const int32_t *__restrict__ bstart, const int32_t *__restrict__ bcount,
                                                     int64_t N, const T *__restrict__ loc, const T *__restrict__ lc,
                                                     T *__restrict__ far) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int P = p * p, ntri = p * (p + 1) / 2;
    T *Ls = reinterpret_cast<T *>(smraw);  // [R][P]
    T *tk = Ls + R * P;                     // [p]: -1 / (2k)
    T *tnm = tk + p;                        // [ntri]: 1 / ((n + m)(n - m)), n >= m + 2
    int b = blockIdx.x;
    for (int e = threadIdx.x; e < R * P; e += L2P_THREADS) Ls[e] = lc[(size_t)b * R * P + e];
    for (int e = threadIdx.x; e < p; e += L2P_THREADS) tk[e] = e > 0 ? (T)(-0.5) / (T)e : (T)0;
    for (int e = threadIdx.x; e < ntri; e += L2P_THREADS) {
        int n = 0;
        while ((n + 1) * (n + 2) / 2 <= e) ++n;
        const int m = e - n * (n + 1) / 2;
        tnm[e] = n >= m + 2 ? (T)1 / ((T)(n + m) * (T)(n - m)) : (T)0;
    }
    __syncthreads();
    int s0 = bstart[b], cnt = bcount[b];
    // each lane evaluates two points at once (c0 and c0 + 32): two independent recurrence chains,
    // and every coefficient read from shared memory serves both
    for (int c0 = threadIdx.x; c0 < cnt; c0 += 2 * L2P_THREADS) {
        const bool two = c0 + L2P_THREADS < cnt;
        const int64_t i0 = s0 + c0, i1 = s0 + (two ? c0 + L2P_THREADS : c0);
        T x[2] = {loc[i0], loc[i1]}, y[2] = {loc[N + i0], loc[N + i1]}, z[2] = {loc[2 * N + i0], loc[2 * N + i1]};
        T r2[2];
        CompSum<T> acc[2][R];
        T mr[2], mi[2];
#pragma unroll
        for (int u = 0; u < 2; ++u) {
            r2[u] = x[u] * x[u] + y[u] * y[u] + z[u] * z[u];
            mr[u] = 1;
            mi[u] = 0;
        }
        for (int m = 0; m < p; ++m) {
            if (m > 0) {
                const T f = tk[m];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    const T nr = f * (x[u] * mr[u] - y[u] * mi[u]), ni = f * (x[u] * mi[u] + y[u] * mr[u]);
                    mr[u] = nr;
                    mi[u] = ni;
                }
            }
            T col[2][R];
#pragma unroll
            for (int u = 0; u < 2; ++u)
#pragma unroll
                for (int r = 0; r < R; ++r) col[u][r] = (T)0;
            // L_n^m against R_n^m = cr + i ci, for both points
            auto term = [&](int n, const T *cr, const T *ci) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const T *Lr = Ls + r * P + n * n;
                    if (m == 0) {
                        const T l0 = Lr[0];
#pragma unroll
                        for (int u = 0; u < 2; ++u) col[u][r] += l0 * cr[u];
                    } else {
                        const T lre = Lr[2 * m - 1], lim = Lr[2 * m];
#pragma unroll
                        for (int u = 0; u < 2; ++u) col[u][r] += (T)2 * (lre * cr[u] - lim * ci[u]);
                    }
                }
            };
            term(m, mr, mi);
            if (m + 1 < p) {
                T p2r[2], p2i[2], p1r[2], p1i[2];
#pragma unroll
                for (int u = 0; u < 2; ++u) {
                    p2r[u] = mr[u];
                    p2i[u] = mi[u];
                    p1r[u] = z[u] * mr[u];
                    p1i[u] = z[u] * mi[u];
                }
                term(m + 1, p1r, p1i);
                for (int n = m + 2; n < p; ++n) {
                    const T d = tnm[tri_idx(n, m)];
                    const T c2 = (T)(2 * n - 1);
                    T cr[2], ci[2];
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        const T c2z = c2 * z[u];
                        cr[u] = (c2z * p1r[u] - r2[u] * p2r[u]) * d;
                        ci[u] = (c2z * p1i[u] - r2[u] * p2i[u]) * d;
                    }
                    term(n, cr, ci);
#pragma unroll
                    for (int u = 0; u < 2; ++u) {
                        p2r[u] = p1r[u];
                        p2i[u] = p1i[u];
                        p1r[u] = cr[u];
                        p1i[u] = ci[u];
                    }
                }
            }
#pragma unroll
            for (int u = 0; u < 2; ++u)
#pragma unroll
                for (int r = 0; r < R; ++r) acc[u][r].add(col[u][r]);
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            far[r * N + i0] = acc[0][r].get();
            if (two) far[r * N + i1] = acc[1][r].get();
        }
    }
}

// FP32 form of k_l2p with packed two-wide arithmetic (add/mul/fma .f32x2): each lane's two
// points are the two halves of every recurrence and sum, so one instruction advances both. The
// tables are stored as broadcast pairs: the local expansion with the real form's factors folded
// in (m = 0: 1; m > 0: 2 Re, -2 Im), -1/(2k), 1/((n+m)(n-m)) and 2n - 1. Same recurrences, same
// column order and the same TwoSum over the columns as k_l2p.
template <int R>
__global__ void __launch_bounds__(L2P_THREADS) k_l2p_x2(int p, const int32_t *__restrict__ bstart,
                                                        const int32_t *__restrict__ bcount, int64_t N,
                                                        const float *__restrict__ loc, const float *__restrict__ lc,
                                                        float *__restrict__ far) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int P = p * p, ntri = p * (p + 1) / 2;
    float2 *Ls = reinterpret_cast<float2 *>(smraw);  // [R][P]
    float2 *tk = Ls + R * P;                          // [p]
    float2 *tnm = tk + p;                             // [ntri]
    float2 *c2t = tnm + ntri;                         // [p]: 2n - 1
    const int b = blockIdx.x;
    for (int e = threadIdx.x; e < R * P; e += L2P_THREADS) {
        const int k = e % P;
        int n = 0;
        while ((n + 1) * (n + 1) <= k) ++n;
        const int j = k - n * n;
        const float f = j == 0 ? 1.f : ((j & 1) ? 2.f : -2.f);
        const float v = f * lc[(size_t)b * R * P + e];
        Ls[e] = make_float2(v, v);
    }
    for (int e = threadIdx.x; e < p; e += L2P_THREADS) {
        const float v = e > 0 ? -0.5f / (float)e : 0.f;
        tk[e] = make_float2(v, v);
        const float c = (float)(2 * e - 1);
        c2t[e] = make_float2(c, c);
    }
    for (int e = threadIdx.x; e < ntri; e += L2P_THREADS) {
        int n = 0;
        while ((n + 1) * (n + 2) / 2 <= e) ++n;
        const int m = e - n * (n + 1) / 2;
        const float v = n >= m + 2 ? 1.f / ((float)(n + m) * (float)(n - m)) : 0.f;
        tnm[e] = make_float2(v, v);
    }
    __syncthreads();
    const int s0 = bstart[b], cnt = bcount[b];
    for (int c0 = threadIdx.x; c0 < cnt; c0 += 2 * L2P_THREADS) {
        const bool two = c0 + L2P_THREADS < cnt;
        const int64_t i0 = s0 + c0, i1 = s0 + (two ? c0 + L2P_THREADS : c0);
        const float2 X = make_float2(loc[i0], loc[i1]), Y = make_float2(loc[N + i0], loc[N + i1]),
                     Z = make_float2(loc[2 * N + i0], loc[2 * N + i1]);
        const float2 NY = make_float2(-Y.x, -Y.y);
        const float2 R2 = __ffma2_rn(Z, Z, __ffma2_rn(Y, Y, __fmul2_rn(X, X)));
        const float2 NR2 = make_float2(-R2.x, -R2.y);
        CompSum<float> acc[2][R];
        float2 MR = make_float2(1.f, 1.f), MI = make_float2(0.f, 0.f);
        for (int m = 0; m < p; ++m) {
            if (m > 0) {
                const float2 F = tk[m];
                const float2 a = __ffma2_rn(X, MR, __fmul2_rn(NY, MI));  // x mr - y mi
                const float2 bb = __ffma2_rn(X, MI, __fmul2_rn(Y, MR));  // x mi + y mr
                MR = __fmul2_rn(F, a);
                MI = __fmul2_rn(F, bb);
            }
            float2 col[R];
#pragma unroll
            for (int r = 0; r < R; ++r) col[r] = make_float2(0.f, 0.f);
            auto term = [&](int n, float2 cr, float2 ci) {
#pragma unroll
                for (int r = 0; r < R; ++r) {
                    const float2 *Lr = Ls + r * P + n * n;
                    if (m == 0) {
                        col[r] = __ffma2_rn(Lr[0], cr, col[r]);
                    } else {
                        col[r] = __ffma2_rn(Lr[2 * m - 1], cr, col[r]);
                        col[r] = __ffma2_rn(Lr[2 * m], ci, col[r]);
                    }
                }
            };
            term(m, MR, MI);
            if (m + 1 < p) {
                float2 P2R = MR, P2I = MI, P1R = __fmul2_rn(Z, MR), P1I = __fmul2_rn(Z, MI);
                term(m + 1, P1R, P1I);
                for (int n = m + 2; n < p; ++n) {
                    const float2 D = tnm[tri_idx(n, m)];
                    const float2 C2Z = __fmul2_rn(c2t[n], Z);
                    const float2 CR = __fmul2_rn(__ffma2_rn(C2Z, P1R, __fmul2_rn(NR2, P2R)), D);
                    const float2 CI = __fmul2_rn(__ffma2_rn(C2Z, P1I, __fmul2_rn(NR2, P2I)), D);
                    term(n, CR, CI);
                    P2R = P1R;
                    P2I = P1I;
                    P1R = CR;
                    P1I = CI;
                }
            }
#pragma unroll
            for (int r = 0; r < R; ++r) {
                acc[0][r].add(col[r].x);
                acc[1][r].add(col[r].y);
            }
        }
#pragma unroll
        for (int r = 0; r < R; ++r) {
            far[r * N + i0] = acc[0][r].get();
            if (two) far[r * N + i1] = acc[1][r].get();
        }
    }
}

template <class T>
__global__ void k_zero(size_t n, T *a) {
    size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    if (i < n) a[i] = (T)0;
}

// out[perm[k]] = (far_k + near_k) / h_leaf: the far field (L2P) and the near field (P2P, run
// concurrently on the side stream) meet here, back in the caller's vertex order.
template <class T>
__global__ void k_combine_out(int64_t N, int R, const int32_t *__restrict__ perm, const T *__restrict__ far,
                              const double *__restrict__ near, const double *__restrict__ ih, RhsArgs<kMaxRhs> a) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= N) return;
    int j = perm[k];
    for (int r = 0; r < R; ++r) a.out[r][j] = ((double)far[r * N + k] + near[r * N + k]) * ih[k];
}

// Chunks of at most `per` pairs within each class.
void make_chunks(const std::vector<int64_t> &class_off, int64_t base, int per, std::vector<XChunk> &out) {
    for (size_t c = 0; c + 1 < class_off.size(); ++c)
        for (int64_t s = class_off[c]; s < class_off[c + 1]; s += per) {
            XChunk ch;
            ch.cls = (int32_t)c;
            ch.start = base + s;
            ch.count = (int32_t)std::min<int64_t>(per, class_off[c + 1] - s);
            out.push_back(ch);
        }
}

template <class T, int R>
void run_fmm(Context &c, const RhsArgs<R> &a, const Operators &opr) {
    Tree &t = c.tree;
    cudaStream_t st = c.stream;
    const int64_t N = c.N;
    const int L = t.L, p = opr.p, P = opr.P;
    const int tb = 256;
    constexpr bool F64 = sizeof(T) == 8;
    T *q, *w, *mp, *lc, *far;
    const T *loc, *nrm;
    const T *m2l, *m2m, *l2l;
    size_t exp_sz = (size_t)t.nbox * R * P;
    if (F64) {
        c.q64.resize((size_t)R * N);
        c.w64.resize((size_t)R * N);
        c.mp64.resize(exp_sz);
        c.lc64.resize(exp_sz);
        c.far64.resize((size_t)R * N);
        q = (T *)c.q64.p; w = (T *)c.w64.p; mp = (T *)c.mp64.p; lc = (T *)c.lc64.p; far = (T *)c.far64.p;
        loc = (const T *)t.loc64.p; nrm = (const T *)t.nrm64.p;
        m2l = (const T *)opr.m2l64.p; m2m = (const T *)opr.m2m64.p; l2l = (const T *)opr.l2l64.p;
    } else {
        c.q32.resize((size_t)R * N);
        c.w32.resize((size_t)R * N);
        c.mp32.resize(exp_sz);
        c.lc32.resize(exp_sz);
        c.far32.resize((size_t)R * N);
        q = (T *)c.q32.p; w = (T *)c.w32.p; mp = (T *)c.mp32.p; lc = (T *)c.lc32.p; far = (T *)c.far32.p;
        loc = (const T *)t.loc32.p; nrm = (const T *)t.nrm32.p;
        m2l = (const T *)opr.m2l32.p; m2m = (const T *)opr.m2m32.p; l2l = (const T *)opr.l2l32.p;
    }
    {
        PhaseScope ps(c, PH_STRENGTHS);
        k_strengths<T, R><<<div_up(N, tb), tb, 0, st>>>(N, t.perm.p, t.s_sorted.p, a, t.ih.p, q, w);
        BEM_LAUNCH_CHECK();
    }
    // The near field needs only the strengths: it runs on the low-priority side stream,
    // overlapped with the whole far field below (the two meet in k_combine_out). P2P keeps the
    // FP32 cores busy while M2L occupies the tensor cores with few warps per SM.
    c.near_out.resize((size_t)R * N);
    if (!c.side) {
        int least = 0, greatest = 0;
        BEM_CUDA(cudaDeviceGetStreamPriorityRange(&least, &greatest));
        BEM_CUDA(cudaStreamCreateWithPriority(&c.side, cudaStreamNonBlocking, least));
        BEM_CUDA(cudaStreamCreateWithPriority(&c.hi, cudaStreamNonBlocking, greatest));
        BEM_CUDA(cudaEventCreateWithFlags(&c.ev_fork, cudaEventDisableTiming));
        BEM_CUDA(cudaEventCreateWithFlags(&c.ev_join, cudaEventDisableTiming));
        BEM_CUDA(cudaEventCreateWithFlags(&c.ev_far, cudaEventDisableTiming));
        BEM_CUDA(cudaEventCreateWithFlags(&c.ev_m2l, cudaEventDisableTiming));
    }
    // overlap mode (c.tuned_overlap): 0 = one stream; 1 = the near field starts with the far
    // field (right after the strengths); 2 = the near field starts when the M2L does: the
    // ALU-bound P2M runs alone, and the near field fills the SMs around the tensor-core M2L's
    // blocks (queued first, on the high-priority stream) and the rest of the far field
    const int omode = c.tuned_overlap;
    const bool ovl = omode != 0;
    cudaStream_t ns = ovl ? c.side : st;  // near-field stream
    BEM_CUDA(cudaEventRecord(c.ev_fork, st));
    bool near_done = false;
    auto launch_near = [&](cudaEvent_t after) {
        if (near_done) return;
        near_done = true;
        if (ovl) BEM_CUDA(cudaStreamWaitEvent(ns, after, 0));
        {
            PhaseScope ps(c, PH_P2P, ns);
            bool hq = false, hw = false;
            for (int r = 0; r < R; ++r) {
                hq = hq || a.f[r] != 0.0;
                hw = hw || a.g[r] != 0.0;
            }
            launch_p2p_list<T, R>(c, q, w, c.near_out.p, hq, hw, ns);
        }
        BEM_CUDA(cudaEventRecord(c.ev_join, ns));
    };
    if (omode != 2) launch_near(c.ev_fork);
    // the far field runs on a high-priority stream, so its blocks (the tensor-core M2L's in
    // particular) are placed as soon as an SM has room and the near field fills the rest
    cudaStream_t fs = ovl ? c.hi : st;
    if (ovl) BEM_CUDA(cudaStreamWaitEvent(fs, c.ev_fork, 0));

    // chunk tables for this R (built once per build)
    const int per = xt_cols<T>() / R;
    auto &mch = c.m2l_chunks_h;
    if (mch.empty() || mch.front().cls != -R) {
        std::vector<XChunk> all;
        XChunk tag{-R, 0, 0};
        all.push_back(tag);  // header: which R the table is for
        make_chunks(t.m2l_class_off, 0, per, all);
        for (int l = 3; l <= L; ++l) make_chunks(t.up_class_off[l], t.up_off[l], per, all);
        mch = all;
        c.m2l_chunks.resize(all.size());
        BEM_CUDA(cudaMemcpyAsync(c.m2l_chunks.p, all.data(), all.size() * sizeof(XChunk), cudaMemcpyHostToDevice, fs));
    }
    // locate the per-phase ranges in the chunk table
    int64_t nm2l_chunks = 0;
    for (size_t cc = 0; cc + 1 < t.m2l_class_off.size(); ++cc)
        nm2l_chunks += (t.m2l_class_off[cc + 1] - t.m2l_class_off[cc] + per - 1) / per;
    std::vector<int64_t> up_first(L + 2, 0), up_n(L + 2, 0);
    int64_t cur = 1 + nm2l_chunks;
    for (int l = 3; l <= L; ++l) {
        int64_t k = 0;
        for (int cc = 0; cc < 8; ++cc) k += (t.up_class_off[l][cc + 1] - t.up_class_off[l][cc] + per - 1) / per;
        up_first[l] = cur;
        up_n[l] = k;
        cur += k;
    }
    const int rowblocks = div_up(P, xt_rows<T>());

    // P2M at the leaves
    const int nleaf = t.nb[L];
    {
        PhaseScope ps(c, PH_P2M, fs);
        const int ntri = p * (p + 1) / 2;
        size_t sm = ((size_t)2 * P2M_PC * ntri + P2M_PC * 3 + 2 * P2M_PC * R + p + ntri) * sizeof(T);
        const int threads = ntri <= 256 ? 128 : 256;  // ntri <= 2 * threads
        bool hw = false;
        for (int r = 0; r < R; ++r) hw = hw || a.g[r] != 0.0;
        if (!F64 && R == 1 && !hw && ntri <= 256) {  // packed FP32x2 form (every GMRES product)
            const size_t smx = (size_t)2 * ntri * P2MX_RS * sizeof(float) + P2M_PC * sizeof(float) +
                               (size_t)(2 * p + ntri) * sizeof(float2);
            if (smx > 48 * 1024)
                BEM_CUDA(cudaFuncSetAttribute(k_p2m_x2, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smx));
            k_p2m_x2<<<nleaf, 128, smx, fs>>>(p, nleaf, t.bstart.p + t.base[L], t.bcount.p + t.base[L], N,
                                              (const float *)loc, (const float *)q,
                                              (float *)mp + (size_t)t.base[L] * P);
        } else {
            auto kern = hw ? k_p2m<T, R, true> : k_p2m<T, R, false>;
            if (sm > 48 * 1024)
                BEM_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm));
            kern<<<nleaf, threads, sm, fs>>>(p, nleaf, t.bstart.p + t.base[L], t.bcount.p + t.base[L], N, loc, nrm, q,
                                             w, mp + (size_t)t.base[L] * R * P);
        }
        BEM_LAUNCH_CHECK();
    }
    // zero the multipoles above the leaves and all locals
    {
        size_t nup = (size_t)t.base[L] * R * P;
        if (nup) k_zero<T><<<div_up(nup, tb), tb, 0, fs>>>(nup, mp);
        k_zero<T><<<div_up(exp_sz, tb), tb, 0, fs>>>(exp_sz, lc);
        BEM_LAUNCH_CHECK();
    }
    // per-pair buffer for the fixed-order reductions
    T *ypair;
    {
        int64_t nup_all = t.up_off[L + 1];
        size_t need = (size_t)std::max<int64_t>(std::max<int64_t>(t.n_m2l, nup_all), 1) * R * P;
        if (F64) {
            c.ypair64.resize(need);
            ypair = (T *)c.ypair64.p;
        } else {
            c.ypair32.resize(need);
            ypair = (T *)c.ypair32.p;
        }
    }
    // M2M upward, levels L -> 2: per-pair products, then each parent sums its children
    for (int l = L; l >= 3; --l) {
        PhaseScope ps(c, PH_M2M, fs);
        if (!up_n[l]) continue;
        dim3 grid((unsigned)up_n[l], rowblocks);
        xlat_smem_attr(k_xlat<T, R, kStorePair>, xt_smem<T>());
        k_xlat<T, R, kStorePair><<<grid, XT_THREADS, xt_smem<T>(), fs>>>(m2m, P, c.m2l_chunks.p + up_first[l],
                                                                         t.up_child.p, t.up_parent.p, mp, ypair, nullptr);
        BEM_LAUNCH_CHECK();
        launch_reduce_pairs<T, R>(t.base[l - 1], t.nb[l - 1], t.up_par_off.p, t.up_by_par.p, ypair, P, mp, fs);
    }
    // M2L, all levels at once, then each target sums its sources
    if (nm2l_chunks) {
        // Single-RHS products (every GMRES product) use the tensor cores with m2l_tensor_cores >= 1;
        // the 4-RHS product behind the diagonals where build decided so (diag_tc): M_ii and L_ii
        // are formed by cancellation (Eqs. (s3), (s5)), which magnifies the far field's rounding.
        const bool tc_path = !F64 && (R == 1 ? c.prm.m2l_tensor_cores >= 1 : R == 4 && c.diag_tc) &&
                             m2l_tc_supported(P) && opr.tc_Npad > 0;
        // target-major (no per-translation rows) for the single-RHS products; the 4-RHS diagonal
        // product stays pair-major (its target-major form, at 64 targets per tile, was slower and
        // less accurate)
        const bool tm_path = tc_path && R == 1 && c.prm.m2l_target_major;
        if (tm_path) {
            PhaseScope ps(c, PH_M2L, fs);
            launch_m2l_tm<1>(c, opr, (const float *)mp, (int64_t)t.nbox, c.tc_err.p, fs);
        } else if (tc_path) {
            PhaseScope ps(c, PH_M2L, fs);
            const int ti = R == 1 ? 0 : 1;
            if (!c.tc_chunks_ok[ti]) {
                // chunk sizes per class: four tiles of rows for small truncated classes, else two
                std::vector<XChunk> tc;
                const int P16 = (P + 15) / 16 * 16;
                for (int cc = 0; cc < kNumM2LClasses; ++cc) {
                    const int Kc = opr.margin >= 0 ? opr.cls_Kh[cc] : P16;
                    const std::vector<int64_t> one = {t.m2l_class_off[cc], t.m2l_class_off[cc + 1]};
                    std::vector<XChunk> part;
                    make_chunks(one, 0, m2l_tc_pairs_per_chunk(R, Kc), part);
                    for (XChunk &x : part) x.cls = cc;
                    tc.insert(tc.end(), part.begin(), part.end());
                }
                c.tc_chunks[ti].resize(std::max<size_t>(tc.size(), 1));
                if (!tc.empty())
                    BEM_CUDA(cudaMemcpyAsync(c.tc_chunks[ti].p, tc.data(), tc.size() * sizeof(XChunk),
                                             cudaMemcpyHostToDevice, fs));
                c.n_tc_chunks[ti] = (int64_t)tc.size();
                c.tc_chunks_ok[ti] = true;
            }
            if (c.n_tc_chunks[ti])
                launch_m2l_tc<R>(c, opr, c.tc_chunks[ti].p, c.n_tc_chunks[ti], (const float *)mp, (int64_t)t.nbox * R,
                                 (float *)ypair, c.tc_err.p, fs);
        } else {
            PhaseScope ps(c, PH_M2L_CC, fs);
            dim3 grid((unsigned)nm2l_chunks, rowblocks);
            xlat_smem_attr(k_xlat<T, R, kStorePair>, xt_smem<T>());
            k_xlat<T, R, kStorePair><<<grid, XT_THREADS, xt_smem<T>(), fs>>>(m2l, P, c.m2l_chunks.p + 1,
                                                                             t.m2l_src.p, t.m2l_tgt.p, mp, ypair,
                                                                             opr.margin >= 0 ? opr.cls_K.p : nullptr);
            BEM_LAUNCH_CHECK();
        }
        if (omode == 2) {  // the M2L is queued: the near field may start (after the multipoles)
            BEM_CUDA(cudaEventRecord(c.ev_m2l, fs));
            launch_near(c.ev_m2l);
        }
        PhaseScope ps(c, PH_M2L_REDUCE, fs);
        if (tm_path) {
            launch_m2l_tm_reduce<1>(c, opr, (float *)lc, fs);
        } else {
            const bool trunc = opr.margin >= 0;
            if (trunc) {
                c.m2l_byK.resize(std::max<int64_t>(t.n_m2l, 1));
                k_pair_K<<<div_up(t.n_m2l, 256), 256, 0, fs>>>(t.n_m2l, t.m2l_by_tgt.p, t.m2l_cls.p, opr.cls_K.p,
                                                              c.m2l_byK.p);
                BEM_LAUNCH_CHECK();
            }
            launch_reduce_pairs<T, R>(t.base[2], t.nbox - t.base[2], t.m2l_tgt_off.p, t.m2l_by_tgt.p, ypair, P, lc,
                                      fs, trunc ? c.m2l_byK.p : nullptr);
        }
    }
    // L2L downward, levels 3 -> L: every child has exactly one parent, so it adds in place
    for (int l = 3; l <= L; ++l) {
        if (!up_n[l]) continue;
        PhaseScope ps(c, PH_L2L, fs);
        dim3 grid((unsigned)up_n[l], rowblocks);
        xlat_smem_attr(k_xlat<T, R, kAddTarget>, xt_smem<T>());
        k_xlat<T, R, kAddTarget><<<grid, XT_THREADS, xt_smem<T>(), fs>>>(l2l, P, c.m2l_chunks.p + up_first[l],
                                                                         t.up_parent.p, t.up_child.p, lc, lc, nullptr);
        BEM_LAUNCH_CHECK();
    }
    // L2P
    {
        PhaseScope ps(c, PH_L2P, fs);
        if constexpr (F64) {
            size_t sm = ((size_t)R * P + p + (size_t)p * (p + 1) / 2) * sizeof(T);  // expansion + divisor tables
            k_l2p<T, R><<<nleaf, L2P_THREADS, sm, fs>>>(p, t.bstart.p + t.base[L], t.bcount.p + t.base[L], N, loc,
                                                        lc + (size_t)t.base[L] * R * P, far);
        } else {  // packed FP32x2: the expansion and the tables as broadcast pairs
            size_t sm = ((size_t)R * P + 2 * p + (size_t)p * (p + 1) / 2) * sizeof(float2);
            k_l2p_x2<R><<<nleaf, L2P_THREADS, sm, fs>>>(p, t.bstart.p + t.base[L], t.bcount.p + t.base[L], N,
                                                        (const float *)loc, (const float *)lc + (size_t)t.base[L] * R * P,
                                                        (float *)far);
        }
        BEM_LAUNCH_CHECK();
    }
    launch_near(c.ev_fork);  // (no M2L pairs: the near field has not started yet)
    BEM_CUDA(cudaEventRecord(c.ev_far, fs));
    // join the near field, add the far field, scale by 1/h and return to the caller's order
    if (ovl) {
        BEM_CUDA(cudaStreamWaitEvent(st, c.ev_far, 0));
        BEM_CUDA(cudaStreamWaitEvent(st, c.ev_join, 0));
    }
    RhsArgs<kMaxRhs> o{};
    for (int r = 0; r < R; ++r) o.out[r] = a.out[r];
    k_combine_out<T><<<div_up(N, tb), tb, 0, st>>>(N, R, t.perm.p, far, c.near_out.p, t.ih.p, o);
    BEM_LAUNCH_CHECK();
}

}  // namespace

// Truncation order of each M2L offset class (see bem_params.m2l_order_margin).
std::vector<int> m2l_class_orders(int p, int margin) {
    std::vector<int> out(kNumM2LClasses, p);
    if (margin < 0) return out;
    const double a = std::sqrt(3.0) / 2.0;  // circumradius of a unit box
    const double rho0 = a / (2.0 - a);      // nearest class, centres 2 boxes apart
    int cidx = 0;
    for (int x = -3; x <= 3; ++x)
        for (int y = -3; y <= 3; ++y)
            for (int z = -3; z <= 3; ++z) {
                if (x >= -1 && x <= 1 && y >= -1 && y <= 1 && z >= -1 && z <= 1) continue;
                const double d = std::sqrt((double)(x * x + y * y + z * z));
                const double rho = a / (d - a);
                const int pc = (int)std::ceil(p * std::log(rho0) / std::log(rho) - 1e-9) + margin;
                out[cidx++] = std::max(1, std::min(p, pc));
            }
    return out;
}

void build_operators(Context &c, Operators &o, int p) {
    const int margin = c.prm.m2l_order_margin;
    if (o.ready && o.p == p && o.margin == margin) return;
    o.margin = margin;
    {
        o.cls_p = m2l_class_orders(p, margin);
        const int Pfull16 = (p * p + 15) / 16 * 16;
        std::vector<int32_t> K(kNumM2LClasses);
        for (int k = 0; k < kNumM2LClasses; ++k)
            K[k] = std::min(Pfull16, (o.cls_p[k] * o.cls_p[k] + 15) / 16 * 16);
        o.cls_K.resize(kNumM2LClasses);
        o.cls_Kh.assign(K.begin(), K.end());
        BEM_CUDA(cudaMemcpyAsync(o.cls_K.p, K.data(), K.size() * sizeof(int32_t), cudaMemcpyHostToDevice, c.stream));
        BEM_CUDA(cudaStreamSynchronize(c.stream));
        if (o.ready && o.p == p) return;  // only the truncation changed
    }
    o.p = p;
    o.P = p * p;
    o.tc_Npad = o.tc_Kpad = 0;  // tensor-core tables follow the operators
    size_t PP = (size_t)o.P * o.P;
    o.m2l64.resize(kNumM2LClasses * PP);
    o.m2l32.resize(kNumM2LClasses * PP);
    o.m2m64.resize(8 * PP);
    o.m2m32.resize(8 * PP);
    o.l2l64.resize(8 * PP);
    o.l2l32.resize(8 * PP);
    size_t sm_m2l = (size_t)2 * (2 * p) * (2 * p + 1) / 2 * sizeof(double);
    size_t sm_up = (size_t)2 * p * (p + 1) / 2 * sizeof(double);
    PhaseScope ps(c, PH_OPERATORS);
    k_build_ops<<<kNumM2LClasses, 256, sm_m2l, c.stream>>>(kOpM2L, p, o.m2l64.p, o.m2l32.p);
    BEM_LAUNCH_CHECK();
    k_build_ops<<<8, 256, sm_up, c.stream>>>(kOpM2M, p, o.m2m64.p, o.m2m32.p);
    BEM_LAUNCH_CHECK();
    k_build_ops<<<8, 256, sm_up, c.stream>>>(kOpL2L, p, o.l2l64.p, o.l2l32.p);
    BEM_LAUNCH_CHECK();
    o.ready = true;
}

template <int R>
static void offdiag_R(Context &c, const double *f, const double *const *xL, const double *g,
                      const double *const *xM, double *const *out, int prec, const Operators &o) {
    RhsArgs<R> a{};
    for (int r = 0; r < R; ++r) {
        a.f[r] = f[r];
        a.g[r] = g[r];
        a.xL[r] = xL[r];
        a.xM[r] = xM[r];
        a.out[r] = out[r];
    }
    if (prec == BEM_PREC_FP64) run_fmm<double, R>(c, a, o);
    else run_fmm<float, R>(c, a, o);
}

void offdiag_apply(Context &c, int R, const double *f, const double *const *xL, const double *g,
                   const double *const *xM, double *const *out, int prec, const Operators *ops) {
    const Operators &o = ops ? *ops : c.ops;
    c.stats.n_apply += 1;
    c.stats.n_apply_rhs += R;
    if (c.prm.mvp == BEM_MVP_DIRECT) {
        if (R == 1) launch_direct<1>(c, prec, f, xL, g, xM, out);
        else if (R == 4) launch_direct<4>(c, prec, f, xL, g, xM, out);
        else fail(BEM_ERR_ARG, "unsupported RHS count");
        return;
    }
    if (R == 1) offdiag_R<1>(c, f, xL, g, xM, out, prec, o);
    else if (R == 4) offdiag_R<4>(c, f, xL, g, xM, out, prec, o);
    else fail(BEM_ERR_ARG, "unsupported RHS count");
}

}  // namespace bem
