// Near field of the FMM (Section 3.7, A^(sparse) X) and the direct all-pairs product
// (Section 3.9, brute force), both with the one-point quadrature kernel of Eq. (ns1):
//   u_i += sum_{j != i} [ q_j / |r_i - r_j| + w_j n_j.(r_i - r_j) / |r_i - r_j|^3 ],
// q_j = f s_j X_L,j / (4 pi), w_j = g s_j X_M,j / (4 pi) (Eqs. (2.13), (3.27)).
//
// FP32 variants keep coordinates accurate by construction: the list kernel works in
// leaf-box units with coordinates relative to each leaf centre (integer box offsets are
// exact in FP32), the direct kernel splits coordinates into hi + lo FP32 pairs. Sums are
// formed per shared-memory tile in FP32 and merged with TwoSum compensation.
#include "internal.h"

namespace bem {
namespace {

constexpr int P2P_THREADS = 128;
constexpr double kInv4Pi = 0.0795774715459476678844418816862571810;

template <class T>
__device__ __forceinline__ T rsqrt_t(T x);
template <>
__device__ __forceinline__ float rsqrt_t<float>(float x) { return rsqrtf(x); }
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

// One block per target leaf. Sources of the (up to 27) neighbour leaves are staged tile by tile
// in shared memory as (x, y, z, q) and (n_x, n_y, n_z, w), positions relative to the target
// leaf's centre in leaf-box units; each thread keeps up to KMAX receivers in registers, so a
// staged source feeds several pairs. The self pair has r^2 = 0 exactly (same coordinates, zero
// offset) and is skipped; the paper's quadrature excludes j = i (Eq. (ns1)).
constexpr int P2P_KMAX = 4;

template <class T, int R>
__global__ void __launch_bounds__(P2P_THREADS) k_p2p_list(
    const int32_t *__restrict__ bstart, const int32_t *__restrict__ bcount, const int32_t *__restrict__ nbr,
    const int32_t *__restrict__ ncnt, const int8_t *__restrict__ nd, int64_t N, const T *__restrict__ loc,
    const T *__restrict__ nrm, const T *__restrict__ q, const T *__restrict__ w, const T *__restrict__ far,
    const double *__restrict__ ih, double *__restrict__ out) {
    using T4 = typename V4<T>::type;
    __shared__ T4 sA[P2P_THREADS];            // x, y, z, q (first RHS)
    __shared__ T4 sB[P2P_THREADS];            // n_x, n_y, n_z, w (first RHS)
    __shared__ T sQ[R > 1 ? R - 1 : 1][P2P_THREADS], sW[R > 1 ? R - 1 : 1][P2P_THREADS];
    __shared__ int nb_start[27], nb_pre[28];
    __shared__ T nb_d[27][3];
    const int b = blockIdx.x, tid = threadIdx.x;
    const int nn = ncnt[b];
    if (tid < nn) {
        int f = nbr[b * 27 + tid];
        nb_start[tid] = bstart[f];
        nb_pre[tid + 1] = bcount[f];
        nb_d[tid][0] = (T)nd[(b * 27 + tid) * 4 + 0];
        nb_d[tid][1] = (T)nd[(b * 27 + tid) * 4 + 1];
        nb_d[tid][2] = (T)nd[(b * 27 + tid) * 4 + 2];
    }
    __syncthreads();
    if (tid == 0) {
        nb_pre[0] = 0;
        for (int k = 0; k < nn; ++k) nb_pre[k + 1] += nb_pre[k];
    }
    __syncthreads();
    const int S = nb_pre[nn];
    const int s0 = bstart[b], cnt = bcount[b];
    for (int rc0 = 0; rc0 < cnt; rc0 += P2P_THREADS * P2P_KMAX) {
        const int kr = min(P2P_KMAX, (cnt - rc0 + P2P_THREADS - 1) / P2P_THREADS);  // uniform in the block
        T xi[P2P_KMAX], yi[P2P_KMAX], zi[P2P_KMAX];
        Comp<T> acc[P2P_KMAX][R];
#pragma unroll
        for (int k = 0; k < P2P_KMAX; ++k) {
            const int li = rc0 + k * P2P_THREADS + tid;
            const int64_t i = s0 + (li < cnt ? li : 0);
            xi[k] = loc[i];
            yi[k] = loc[N + i];
            zi[k] = loc[2 * N + i];
        }
        for (int t0 = 0; t0 < S; t0 += P2P_THREADS) {
            __syncthreads();
            const int f = t0 + tid;
            if (f < S) {
                int k = 0;
                while (nb_pre[k + 1] <= f) ++k;
                const int j = nb_start[k] + (f - nb_pre[k]);
                sA[tid] = T4{loc[j] + nb_d[k][0], loc[N + j] + nb_d[k][1], loc[2 * N + j] + nb_d[k][2], q[j]};
                sB[tid] = T4{nrm[j], nrm[N + j], nrm[2 * N + j], w[j]};
#pragma unroll
                for (int r = 1; r < R; ++r) {
                    sQ[r - 1][tid] = q[r * N + j];
                    sW[r - 1][tid] = w[r * N + j];
                }
            }
            __syncthreads();
            const int ns = min(P2P_THREADS, S - t0);
            T part[P2P_KMAX][R];
#pragma unroll
            for (int k = 0; k < P2P_KMAX; ++k)
#pragma unroll
                for (int r = 0; r < R; ++r) part[k][r] = (T)0;
#pragma unroll 2
            for (int sI = 0; sI < ns; ++sI) {
                const T4 a = sA[sI], bb = sB[sI];
#pragma unroll
                for (int k = 0; k < P2P_KMAX; ++k) {
                    if (k < kr) {
                        const T dx = xi[k] - a.x, dy = yi[k] - a.y, dz = zi[k] - a.z;
                        const T r2 = dx * dx + dy * dy + dz * dz;
                        const T rinv = r2 > (T)0 ? rsqrt_t<T>(r2) : (T)0;
                        const T rinv3 = rinv * rinv * rinv;
                        const T nd3 = (bb.x * dx + bb.y * dy + bb.z * dz) * rinv3;
                        part[k][0] += a.w * rinv + bb.w * nd3;
#pragma unroll
                        for (int r = 1; r < R; ++r) part[k][r] += sQ[r - 1][sI] * rinv + sW[r - 1][sI] * nd3;
                    }
                }
            }
#pragma unroll
            for (int k = 0; k < P2P_KMAX; ++k)
#pragma unroll
                for (int r = 0; r < R; ++r) acc[k][r].add(part[k][r]);
        }
#pragma unroll
        for (int k = 0; k < P2P_KMAX; ++k) {
            const int li = rc0 + k * P2P_THREADS + tid;
            if (k < kr && li < cnt) {
                const int64_t i = s0 + li;
#pragma unroll
                for (int r = 0; r < R; ++r) out[r * N + i] = ((double)far[r * N + i] + acc[k][r].get()) * ih[i];
            }
        }
    }
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

template <class T, int R>
void launch_p2p_list(Context &c, const T *q, const T *w, const T *far, double *out_sorted) {
    Tree &t = c.tree;
    const int L = t.L;
    const T *loc = sizeof(T) == 8 ? (const T *)t.loc64.p : (const T *)t.loc32.p;
    const T *nrm = sizeof(T) == 8 ? (const T *)t.nrm64.p : (const T *)t.nrm32.p;
    int nleaf = t.nb[L];
    k_p2p_list<T, R><<<nleaf, P2P_THREADS, 0, c.stream>>>(t.bstart.p + t.base[L], t.bcount.p + t.base[L], t.nbr.p,
                                                          t.nbr_cnt.p, t.nbr_d.p, c.N, loc, nrm, q, w, far, t.ih.p,
                                                          out_sorted);
    BEM_LAUNCH_CHECK();
}

template void launch_p2p_list<float, 1>(Context &, const float *, const float *, const float *, double *);
template void launch_p2p_list<float, 4>(Context &, const float *, const float *, const float *, double *);
template void launch_p2p_list<double, 1>(Context &, const double *, const double *, const double *, double *);
template void launch_p2p_list<double, 4>(Context &, const double *, const double *, const double *, double *);

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
