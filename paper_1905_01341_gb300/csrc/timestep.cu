// Time step of the bubble-dynamics method (Sections 3.4-3.6) on the device:
//   - spherical shape filter x_hat = G (G^(-1) x) per bubble (Eqs. (3.22)-(3.25)), applied to
//     the inputs (r, phi) and to the outputs (dr/dt, dphi/dt) of every right-hand side;
//   - Dirichlet solve for q through the FMM/GMRES path of this library;
//   - tangential velocity from Stokes' theorem (Eqs. (3.7)-(3.11));
//   - mean curvature from the paraboloid through five neighbours (Eqs. (parab1)-(parab2));
//   - bubble volume (divergence theorem on the facets) and polytropic gas (Eq. (2.8));
//   - dr/dt = v + alpha v_t = n q and dphi/dt = (alpha v_t + v/2).v - (p_g - 2 sigma H) + F(t)
//     with alpha = -1, F(t) = 1 - Pa sin(omega t) (Eqs. (2.6), (3.13)-(3.15));
//   - 4th-order Runge-Kutta for the first five steps, then 6th-order Adams-Bashforth
//     (Section 3.5), constant dt from Eq. (3.12).
// All arithmetic is FP64. Per-vertex sums run over the sorted vertex->triangle lists and
// per-bubble sums are block reductions in a fixed order, so a step is reproducible.
#include "internal.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>

namespace bem {

constexpr int kGuessMax = 3;        // highest degree of the extrapolated initial guess
constexpr int kQh = kGuessMax + 1;  // step-start solutions kept for it

// Section 3.5's schemes. Adams-Bashforth of order k: y_{n+1} = y_n + dt sum_j b_j f_{n-j}
// (newest first); Adams-Moulton corrector of order k: y_{n+1} = y_n + dt sum_j m_j f_{n+1-j}
// (f_{n+1} first, at the predicted state); Runge-Kutta starts of order 4 (classical), 5
// (Butcher's six-stage method) and 6 (Butcher's seven-stage method with rational coefficients).
constexpr double kAB[6][6] = {
    {1.0},
    {3.0 / 2.0, -1.0 / 2.0},
    {23.0 / 12.0, -16.0 / 12.0, 5.0 / 12.0},
    {55.0 / 24.0, -59.0 / 24.0, 37.0 / 24.0, -9.0 / 24.0},
    {1901.0 / 720.0, -2774.0 / 720.0, 2616.0 / 720.0, -1274.0 / 720.0, 251.0 / 720.0},
    {4277.0 / 1440.0, -7923.0 / 1440.0, 9982.0 / 1440.0, -7298.0 / 1440.0, 2877.0 / 1440.0, -475.0 / 1440.0}};
constexpr double kAM[3][6] = {  // orders 4, 5, 6
    {9.0 / 24.0, 19.0 / 24.0, -5.0 / 24.0, 1.0 / 24.0},
    {251.0 / 720.0, 646.0 / 720.0, -264.0 / 720.0, 106.0 / 720.0, -19.0 / 720.0},
    {475.0 / 1440.0, 1427.0 / 1440.0, -798.0 / 1440.0, 482.0 / 1440.0, -173.0 / 1440.0, 27.0 / 1440.0}};
struct Tableau {
    int s;
    double c[7], a[7][7], b[7];
};
const Tableau kRK[3] = {
    {4, {0.0, 0.5, 0.5, 1.0}, {{0}, {0.5}, {0.0, 0.5}, {0.0, 0.0, 1.0}}, {1.0 / 6.0, 2.0 / 6.0, 2.0 / 6.0, 1.0 / 6.0}},
    {6,
     {0.0, 0.25, 0.25, 0.5, 0.75, 1.0},
     {{0}, {0.25}, {0.125, 0.125}, {0.0, -0.5, 1.0}, {3.0 / 16.0, 0.0, 0.0, 9.0 / 16.0},
      {-3.0 / 7.0, 2.0 / 7.0, 12.0 / 7.0, -12.0 / 7.0, 8.0 / 7.0}},
     {7.0 / 90.0, 0.0, 32.0 / 90.0, 12.0 / 90.0, 32.0 / 90.0, 7.0 / 90.0}},
    {7,
     {0.0, 1.0 / 3.0, 2.0 / 3.0, 1.0 / 3.0, 0.5, 0.5, 1.0},
     {{0}, {1.0 / 3.0}, {0.0, 2.0 / 3.0}, {1.0 / 12.0, 1.0 / 3.0, -1.0 / 12.0},
      {-1.0 / 16.0, 9.0 / 8.0, -3.0 / 16.0, -3.0 / 8.0}, {0.0, 9.0 / 8.0, -3.0 / 8.0, -3.0 / 4.0, 0.5},
      {9.0 / 44.0, -9.0 / 11.0, 63.0 / 44.0, 18.0 / 11.0, 0.0, -16.0 / 11.0}},
     {11.0 / 120.0, 0.0, 81.0 / 120.0, 81.0 / 120.0, -32.0 / 120.0, -32.0 / 120.0, 11.0 / 120.0}}};

struct StepState {
    bool ready = false;
    bem_step_params sp{};
    double t = 0.0, dt = 0.0;
    int64_t steps = 0;
    int nhist = 0;  // valid history entries (newest at index 0 of `order`)
    int order[5] = {0, 1, 2, 3, 4};
    int Pf = 0;
    DevBuf<double> y, q, hist, ks[7], ytmp, yf, f, fp;
    DevBuf<double> fio;  // host-side arguments of bem_step_filter, staged
    DevBuf<double> V0, a0, V, pg;
    DevBuf<int32_t> bub_of, nbr5;
    DevBuf<int64_t> voff, toff;
    ShBasis filt;  // shape filter basis (bandwidth p_f)
    DevBuf<double> x0;  // r at t = 0 (SoA)
    DevBuf<double> vt, H;
    bem_step_stats last{};
    // q of the last kQh step-start solves (newest first through qh_order) and their times, for
    // the extrapolated initial guess
    DevBuf<double> qh;  // [kQh][N]
    double qh_time[kQh] = {};  // per slot
    int qh_order[kQh] = {0, 1, 2, 3};
    int qh_n = 0;
};

namespace {

constexpr double kPi = 3.14159265358979323846;
constexpr int kMaxNbrCand = 64;

StepState &state_of(Context &c) {
    if (!c.step) c.step = new StepState();
    return *c.step;
}

// Five lowest-index neighbours (vertices sharing an edge) of every vertex.
__global__ void k_nbr5(int64_t N, int64_t T, const int32_t *__restrict__ tri, const int32_t *__restrict__ off,
                       const int32_t *__restrict__ v2t, int32_t *__restrict__ nbr5, int *__restrict__ bad) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= N) return;
    int cand[kMaxNbrCand];
    int n = 0;
    for (int t = off[j]; t < off[j + 1]; ++t) {
        int64_t k = v2t[t];
        for (int c = 0; c < 3; ++c) {
            int v = tri[c * T + k];
            if (v == (int)j) continue;
            bool dup = false;
            for (int i = 0; i < n; ++i) dup |= (cand[i] == v);
            if (!dup && n < kMaxNbrCand) cand[n++] = v;
        }
    }
    if (n < 5) {
        atomicOr(bad, 1);
        for (int i = 0; i < 5; ++i) nbr5[j * 5 + i] = (int)j;
        return;
    }
    // partial selection of the five smallest
    for (int i = 0; i < 5; ++i) {
        int mi = i;
        for (int k = i + 1; k < n; ++k)
            if (cand[k] < cand[mi]) mi = k;
        int tmp = cand[i];
        cand[i] = cand[mi];
        cand[mi] = tmp;
        nbr5[j * 5 + i] = cand[i];
    }
}

// Fully normalised real spherical harmonics (orthonormal on the unit sphere) of degrees
// 0..pf-1 at one unit direction; column order j = n^2 + n + m.
__device__ void real_sh_row(double dx, double dy, double dz, int pf, double *out, double *pb) {
    double len = sqrt(dx * dx + dy * dy + dz * dz);
    double ct = fmin(fmax(dz / len, -1.0), 1.0);
    double st = sqrt(fmax(0.0, 1.0 - ct * ct));
    double ph = atan2(dy, dx);
    // pb[n * pf + m]
    pb[0] = sqrt(1.0 / (4.0 * kPi));
    for (int m = 1; m < pf; ++m) pb[m * pf + m] = -sqrt((2.0 * m + 1.0) / (2.0 * m)) * st * pb[(m - 1) * pf + (m - 1)];
    for (int m = 0; m + 1 < pf; ++m) pb[(m + 1) * pf + m] = sqrt(2.0 * m + 3.0) * ct * pb[m * pf + m];
    for (int m = 0; m < pf; ++m)
        for (int n = m + 2; n < pf; ++n) {
            double a = sqrt((4.0 * n * n - 1.0) / ((double)n * n - (double)m * m));
            double b = sqrt(((n - 1.0) * (n - 1.0) - (double)m * m) / (4.0 * (n - 1.0) * (n - 1.0) - 1.0));
            pb[n * pf + m] = a * (ct * pb[(n - 1) * pf + m] - b * pb[(n - 2) * pf + m]);
        }
    const double r2 = sqrt(2.0);
    for (int n = 0; n < pf; ++n)
        for (int m = -n; m <= n; ++m) {
            int j = n * n + n + m;
            if (m == 0) out[j] = pb[n * pf];
            else if (m > 0) out[j] = r2 * pb[n * pf + m] * cos(m * ph);
            else out[j] = r2 * pb[n * pf - m] * sin(-m * ph);
        }
}

// G[i][*] for the unit directions of one shape (from its representative bubble).
__global__ void k_filter_G(int nd, const double *__restrict__ xyz, int64_t N, int64_t v0, double cx, double cy,
                           double cz, int pf, int ld, double *__restrict__ G, double *__restrict__ scratch) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nd) return;
    int64_t j = v0 + i;
    real_sh_row(xyz[j] - cx, xyz[N + j] - cy, xyz[2 * N + j] - cz, pf, G + (size_t)i * ld,
                scratch + (size_t)i * pf * pf);
}

// Gp = (G^T G)^(-1) G^T by Cholesky (one block) for the first P columns of G (rows of length
// ld); rows P..ld-1 of Gp are zero. A: scratch [P][P].
__global__ void k_filter_pinv(int nd, int P, int ld, const double *__restrict__ G, double *__restrict__ A,
                              double *__restrict__ Gp, int *__restrict__ bad) {
    for (int e = threadIdx.x; e < P * P; e += blockDim.x) {
        int a = e / P, b = e % P;
        double s = 0.0;
        for (int i = 0; i < nd; ++i) s += G[(size_t)i * ld + a] * G[(size_t)i * ld + b];
        A[e] = s;
    }
    for (size_t e = threadIdx.x; e < (size_t)(ld - P) * nd; e += blockDim.x) Gp[(size_t)P * nd + e] = 0.0;
    __syncthreads();
    if (threadIdx.x == 0) {  // in-place Cholesky, lower triangle
        for (int k = 0; k < P; ++k) {
            double d = A[k * P + k];
            for (int m = 0; m < k; ++m) d -= A[k * P + m] * A[k * P + m];
            if (!(d > 0.0)) {
                atomicOr(bad, 4);
                d = 1.0;
            }
            d = sqrt(d);
            A[k * P + k] = d;
            for (int i = k + 1; i < P; ++i) {
                double s = A[i * P + k];
                for (int m = 0; m < k; ++m) s -= A[i * P + m] * A[k * P + m];
                A[i * P + k] = s / d;
            }
        }
    }
    __syncthreads();
    // columns i of G^T: solve L L^T x = G[i][:], write Gp[:][i]
    for (int i = threadIdx.x; i < nd; i += blockDim.x) {
        double x[128];
        for (int a = 0; a < P; ++a) {
            double s = G[(size_t)i * ld + a];
            for (int m = 0; m < a; ++m) s -= A[a * P + m] * x[m];
            x[a] = s / A[a * P + a];
        }
        for (int a = P - 1; a >= 0; --a) {
            double s = x[a];
            for (int m = a + 1; m < P; ++m) s -= A[m * P + a] * x[m];
            x[a] = s / A[a * P + a];
        }
        for (int a = 0; a < P; ++a) Gp[(size_t)a * nd + i] = x[a];
    }
}

// Y = G (Gp X) per bubble for the four SoA components of a state [4N]; may run in place.
__global__ void k_filter_apply(int64_t N, const int64_t *__restrict__ voff, const int32_t *__restrict__ shape_of,
                               const int64_t *__restrict__ g_off, int P, const double *__restrict__ G,
                               const double *__restrict__ Gp, const double *X, double *Y) {
    extern __shared__ double C[];  // [P][4]
    int m = blockIdx.x;
    int64_t a = voff[m];
    int nd = (int)(voff[m + 1] - a);
    const double *Gm = G + g_off[shape_of[m]];
    const double *Gpm = Gp + g_off[shape_of[m]];
    for (int e = threadIdx.x; e < P * 4; e += blockDim.x) {
        int p = e >> 2, comp = e & 3;
        const double *x = X + comp * N + a;
        const double *g = Gpm + (size_t)p * nd;
        double s = 0.0;
        for (int i = 0; i < nd; ++i) s = fma(g[i], x[i], s);
        C[e] = s;
    }
    __syncthreads();
    for (int i = threadIdx.x; i < nd; i += blockDim.x) {
        const double *g = Gm + (size_t)i * P;
        double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
        for (int p = 0; p < P; ++p) {
            double gv = g[p];
            s0 = fma(gv, C[p * 4 + 0], s0);
            s1 = fma(gv, C[p * 4 + 1], s1);
            s2 = fma(gv, C[p * 4 + 2], s2);
            s3 = fma(gv, C[p * 4 + 3], s3);
        }
        Y[a + i] = s0;
        Y[N + a + i] = s1;
        Y[2 * N + a + i] = s2;
        Y[3 * N + a + i] = s3;
    }
}

// The same filter in compensated FP32 arithmetic (mixed precision; FP64 runs at a small fraction
// of the FP32 rate on this part): G and G+ stored as (hi, lo) FP32 pairs, G transposed to
// [P][nd] so that both phases read rows of consecutive vertices; the bubble's fields are split
// the same way as they are staged (FD_CHUNK vertices at a time); every dot product is a TwoProd
// (with the two cross terms) into a TwoSum-compensated sum: about 48 bits, far below any
// tolerance of the time step. Phase 1 (c = G+ x): warp w owns the rows p = w, w + FD_WARPS, ...
// (FD_ROWS per pass) with all four fields, its lanes striding over the vertices, joined by a
// fixed butterfly; phase 2 (x^ = G c): one thread per vertex, four compensated sums.
constexpr int FD_THREADS = 256, FD_WARPS = FD_THREADS / 32, FD_ROWS = 5, FD_CHUNK = 256;

__device__ __forceinline__ void cdot_add(float &s, float &c, float2 g, float2 x) {
    const float p = g.x * x.x;
    float e = fmaf(g.x, x.x, -p);  // exact error of the leading product
    e = fmaf(g.x, x.y, e);
    e = fmaf(g.y, x.x, e);
    const float t = s + p, bp = t - s;
    c += ((s - (t - bp)) + (p - bp)) + e;
    s = t;
}

__device__ __forceinline__ float2 split_df(double v) {
    const float h = (float)v;
    return make_float2(h, (float)(v - (double)h));
}

// b[p * nd + i] = a[i * P + p] (transpose = true) or b[e] = a[e], as (hi, lo) pairs.
__global__ void k_split_df(int64_t nd, int P, bool transpose, const double *__restrict__ a,
                           float2 *__restrict__ b) {
    const int64_t n = nd * P;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        b[e] = split_df(transpose ? a[(e % nd) * P + e / nd] : a[e]);
}

__global__ void __launch_bounds__(FD_THREADS) k_filter_apply_df(int64_t N, const int64_t *__restrict__ voff,
                                                                const int32_t *__restrict__ shape_of,
                                                                const int64_t *__restrict__ g_off, int P,
                                                                const float2 *__restrict__ GT,
                                                                const float2 *__restrict__ Gp, const double *X,
                                                                double *Y) {
    extern __shared__ float2 fsm[];
    float2 *xs = fsm;                 // [4][FD_CHUNK] the fields, split
    float2 *C = fsm + 4 * FD_CHUNK;   // [P][4] the coefficients, (sum, compensation)
    const int m = blockIdx.x;
    const int64_t a = voff[m];
    const int nd = (int)(voff[m + 1] - a);
    const float2 *GTm = GT + g_off[shape_of[m]];
    const float2 *Gpm = Gp + g_off[shape_of[m]];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    for (int r0 = 0; r0 < P; r0 += FD_WARPS * FD_ROWS) {
        float s[FD_ROWS][4], cc[FD_ROWS][4];
#pragma unroll
        for (int r = 0; r < FD_ROWS; ++r)
#pragma unroll
            for (int k = 0; k < 4; ++k) s[r][k] = cc[r][k] = 0.f;
        for (int c0 = 0; c0 < nd; c0 += FD_CHUNK) {
            const int len = min(FD_CHUNK, nd - c0);
            __syncthreads();
            for (int e = tid; e < 4 * FD_CHUNK; e += FD_THREADS) {
                const int comp = e / FD_CHUNK, t = e % FD_CHUNK;
                if (t < len) xs[e] = split_df(X[comp * N + a + c0 + t]);
            }
            __syncthreads();
#pragma unroll 2
            for (int t = lane; t < len; t += 32) {
                float2 g[FD_ROWS];
#pragma unroll
                for (int r = 0; r < FD_ROWS; ++r) {
                    const int p = r0 + warp + r * FD_WARPS;
                    g[r] = p < P ? Gpm[(size_t)p * nd + c0 + t] : make_float2(0.f, 0.f);
                }
#pragma unroll
                for (int k = 0; k < 4; ++k) {
                    const float2 x = xs[k * FD_CHUNK + t];
#pragma unroll
                    for (int r = 0; r < FD_ROWS; ++r) cdot_add(s[r][k], cc[r][k], g[r], x);
                }
            }
        }
#pragma unroll
        for (int r = 0; r < FD_ROWS; ++r) {
            const int p = r0 + warp + r * FD_WARPS;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                float sj = s[r][k], cj = cc[r][k];
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) {
                    const float os = __shfl_xor_sync(0xffffffffu, sj, o), oc = __shfl_xor_sync(0xffffffffu, cj, o);
                    const float t = sj + os, bp = t - sj;
                    cj += ((sj - (t - bp)) + (os - bp)) + oc;
                    sj = t;
                }
                if (lane == 0 && p < P) C[p * 4 + k] = make_float2(sj, cj);
            }
        }
    }
    __syncthreads();
    for (int i = tid; i < nd; i += FD_THREADS) {
        float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f, c0 = 0.f, c1 = 0.f, c2 = 0.f, c3 = 0.f;
#pragma unroll 4
        for (int p = 0; p < P; ++p) {
            const float2 gv = GTm[(size_t)p * nd + i];
            cdot_add(s0, c0, gv, C[p * 4 + 0]);
            cdot_add(s1, c1, gv, C[p * 4 + 1]);
            cdot_add(s2, c2, gv, C[p * 4 + 2]);
            cdot_add(s3, c3, gv, C[p * 4 + 3]);
        }
        Y[a + i] = (double)s0 + (double)c0;
        Y[N + a + i] = (double)s1 + (double)c1;
        Y[2 * N + a + i] = (double)s2 + (double)c2;
        Y[3 * N + a + i] = (double)s3 + (double)c3;
    }
}

// Eq. (3.11) per triangle: (n x v)_k A_k = [(r2 - r3) phi1 + (r3 - r1) phi2 + (r1 - r2) phi3] / 2,
// stored as the pairs (x, y), (z, 0); computed once per triangle instead of once per corner.
__global__ void k_tri_nxv(int64_t T, int64_t N, const double *__restrict__ xyz, const double *__restrict__ phi,
                          const int32_t *__restrict__ tri, double2 *__restrict__ w) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= T) return;
    const double *X = xyz, *Y = xyz + N, *Z = xyz + 2 * N;
    const int a = tri[k], b = tri[T + k], c = tri[2 * T + k];
    const double pa = phi[a], pb = phi[b], pc = phi[c];
    const double wx = 0.5 * ((X[b] - X[c]) * pa + (X[c] - X[a]) * pb + (X[a] - X[b]) * pc);
    const double wy = 0.5 * ((Y[b] - Y[c]) * pa + (Y[c] - Y[a]) * pb + (Y[a] - Y[b]) * pc);
    const double wz = 0.5 * ((Z[b] - Z[c]) * pa + (Z[c] - Z[a]) * pb + (Z[a] - Z[b]) * pc);
    w[2 * k] = make_double2(wx, wy);
    w[2 * k + 1] = make_double2(wz, 0.0);
}

// Eqs. (3.10)-(3.11): v_t,j = (n x v)_j x n_j with (n x v)_j = (1/(3 s_j)) sum_k (n x v)_k A_k over
// the vertex's triangles in vertex-to-triangle list order.
__global__ void k_tangential(int64_t N, const double2 *__restrict__ w, const int32_t *__restrict__ off,
                             const int32_t *__restrict__ v2t, const double *__restrict__ s,
                             const double *__restrict__ nrm, double *__restrict__ vt) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= N) return;
    double ax = 0, ay = 0, az = 0;
    for (int t = off[j]; t < off[j + 1]; ++t) {
        const int64_t k = v2t[t];
        const double2 u = w[2 * k], v = w[2 * k + 1];
        ax += u.x;
        ay += u.y;
        az += v.x;
    }
    double inv = 1.0 / (3.0 * s[j]);
    ax *= inv;
    ay *= inv;
    az *= inv;
    double nx = nrm[j], ny = nrm[N + j], nz = nrm[2 * N + j];
    vt[j] = ay * nz - az * ny;
    vt[N + j] = az * nx - ax * nz;
    vt[2 * N + j] = ax * ny - ay * nx;
}

// Column c of the elimination of the 5 x 6 system [A | z] of k_curvature: partial pivoting
// (the row swap as selects), one reciprocal of the pivot, the rows below updated.
template <int c>
__device__ __forceinline__ void curv_elim_step(double (&A)[5][6], double (&rp)[5], bool &singular) {
    int piv = c;
    double best = fabs(A[c][c]);
#pragma unroll
    for (int r = c + 1; r < 5; ++r)
        if (fabs(A[r][c]) > best) {
            best = fabs(A[r][c]);
            piv = r;
        }
#pragma unroll
    for (int r = c + 1; r < 5; ++r) {
        const bool sw = piv == r;
#pragma unroll
        for (int k = c; k < 6; ++k) {
            const double a = A[c][k], b = A[r][k];
            A[c][k] = sw ? b : a;
            A[r][k] = sw ? a : b;
        }
    }
    singular = singular || A[c][c] == 0.0;
    rp[c] = 1.0 / A[c][c];
#pragma unroll
    for (int r = c + 1; r < 5; ++r) {
        const double f = A[r][c] * rp[c];
#pragma unroll
        for (int k = c + 1; k < 6; ++k) A[r][k] -= f * A[c][k];
    }
}

// Eqs. (parab1)-(parab2): 5x5 interpolation in the frame (e1, e2, n_j); H = -B3 - B5.
// Gaussian elimination with partial pivoting (same solution as Cramer's rule).
__global__ void k_curvature(int64_t N, const double *__restrict__ xyz, const double *__restrict__ nrm,
                            const int32_t *__restrict__ nbr5, double *__restrict__ H, int *__restrict__ bad) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= N) return;
    double n[3] = {nrm[j], nrm[N + j], nrm[2 * N + j]};
    // e1: the coordinate axis least aligned with n, made orthogonal to n
    int ax = 0;
    double amin = fabs(n[0]);
    if (fabs(n[1]) < amin) {
        ax = 1;
        amin = fabs(n[1]);
    }
    if (fabs(n[2]) < amin) ax = 2;
    double e1[3] = {ax == 0 ? 1.0 : 0.0, ax == 1 ? 1.0 : 0.0, ax == 2 ? 1.0 : 0.0};
    double dn = e1[0] * n[0] + e1[1] * n[1] + e1[2] * n[2];
#pragma unroll
    for (int d = 0; d < 3; ++d) e1[d] -= dn * n[d];
    double l1 = sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
#pragma unroll
    for (int d = 0; d < 3; ++d) e1[d] /= l1;
    double e2[3] = {n[1] * e1[2] - n[2] * e1[1], n[2] * e1[0] - n[0] * e1[2], n[0] * e1[1] - n[1] * e1[0]};
    double A[5][6];
#pragma unroll
    for (int l = 0; l < 5; ++l) {
        int k = nbr5[j * 5 + l];
        double d[3] = {xyz[k] - xyz[j], xyz[N + k] - xyz[N + j], xyz[2 * N + k] - xyz[2 * N + j]};
        double x = d[0] * e1[0] + d[1] * e1[1] + d[2] * e1[2];
        double y = d[0] * e2[0] + d[1] * e2[1] + d[2] * e2[2];
        double z = d[0] * n[0] + d[1] * n[1] + d[2] * n[2];
        A[l][0] = x;
        A[l][1] = y;
        A[l][2] = x * x;
        A[l][3] = x * y;
        A[l][4] = y * y;
        A[l][5] = z;
    }
    // Gaussian elimination with partial pivoting, one step per column instantiated at compile
    // time so that the system stays in registers
    double rp[5];
    bool singular = false;
    curv_elim_step<0>(A, rp, singular);
    curv_elim_step<1>(A, rp, singular);
    curv_elim_step<2>(A, rp, singular);
    curv_elim_step<3>(A, rp, singular);
    curv_elim_step<4>(A, rp, singular);
    if (singular) {
        atomicOr(bad, 8);
        H[j] = 0.0;
        return;
    }
    double B[5];
#pragma unroll
    for (int r = 4; r >= 0; --r) {
        double s = A[r][5];
#pragma unroll
        for (int k = r + 1; k < 5; ++k) s -= A[r][k] * B[k];
        B[r] = s * rp[r];
    }
    H[j] = -B[2] - B[4];
}

// V_m = (1/3) sum_k (N_k A_k) . c_k over the bubble's triangles (one block per bubble).
__global__ void k_volumes(int64_t N, int64_t T, const int64_t *__restrict__ toff, const int32_t *__restrict__ tri,
                          const double *__restrict__ xyz, double *__restrict__ V) {
    __shared__ double red[256];
    int m = blockIdx.x;
    const double *X = xyz, *Y = xyz + N, *Z = xyz + 2 * N;
    double acc = 0.0;
    for (int64_t k = toff[m] + threadIdx.x; k < toff[m + 1]; k += blockDim.x) {
        int a = tri[k], b = tri[T + k], c = tri[2 * T + k];
        double e1x = X[b] - X[a], e1y = Y[b] - Y[a], e1z = Z[b] - Z[a];
        double e2x = X[c] - X[a], e2y = Y[c] - Y[a], e2z = Z[c] - Z[a];
        // 2 N_k A_k . 3 c_k; the constant factor 1/18 is applied once to the bubble's sum
        double nx2 = e1y * e2z - e1z * e2y, ny2 = e1z * e2x - e1x * e2z, nz2 = e1x * e2y - e1y * e2x;
        acc += nx2 * (X[a] + X[b] + X[c]) + ny2 * (Y[a] + Y[b] + Y[c]) + nz2 * (Z[a] + Z[b] + Z[c]);
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) V[m] = red[0] / 18.0;
}

__global__ void k_init_bubbles(int M, const double *__restrict__ V, double *__restrict__ V0, double *__restrict__ a0) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    V0[m] = V[m];
    a0[m] = cbrt(3.0 * V[m] / (4.0 * kPi));
}

// Eq. (2.8): p_g = (1 + 2 sigma / a_m0) (V_m0 / V_m)^kappa.
__global__ void k_pressure(int M, const double *__restrict__ V, const double *__restrict__ V0,
                           const double *__restrict__ a0, double sigma, double kappa, double *__restrict__ pg) {
    int m = blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= M) return;
    pg[m] = (1.0 + 2.0 * sigma / a0[m]) * pow(V0[m] / V[m], kappa);
}

__global__ void k_bubble_of(int M, const int64_t *__restrict__ voff, int32_t *__restrict__ bub) {
    int m = blockIdx.x;
    for (int64_t j = voff[m] + threadIdx.x; j < voff[m + 1]; j += blockDim.x) bub[j] = m;
}

// Eqs. (3.13)-(3.15) with alpha = -1: f = [n q ; (alpha v_t + v/2).v - (p_g - 2 sigma H) + F].
__global__ void k_assemble(int64_t N, const double *__restrict__ q, const double *__restrict__ nrm,
                           const double *__restrict__ vt, const double *__restrict__ H, const double *__restrict__ pg,
                           const int32_t *__restrict__ bub, double sigma, double F, double *__restrict__ f) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= N) return;
    const double alpha = -1.0;
    double vt3[3] = {vt[j], vt[N + j], vt[2 * N + j]};
    double v3[3], u3[3];
    for (int d = 0; d < 3; ++d) {
        v3[d] = nrm[d * N + j] * q[j] + vt3[d];
        u3[d] = v3[d] + alpha * vt3[d];
        f[d * N + j] = u3[d];
    }
    double e = 0.0;
    for (int d = 0; d < 3; ++d) e += (alpha * vt3[d] + 0.5 * v3[d]) * v3[d];
    f[3 * N + j] = e - (pg[bub[j]] - 2.0 * sigma * H[j]) + F;
}

// out = y + dt * sum_j w_j f_j (j = 0 .. n-1, in order); out may alias y
struct LinTerms {
    const double *f[7];
    double w[7];
    int n;
};
__global__ void k_lincomb(int64_t len, double dt, const double *__restrict__ y, LinTerms t, double *out) {
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < len; i += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int k = 0; k < t.n; ++k) acc += t.w[k] * t.f[k][i];
        out[i] = y[i] + dt * acc;
    }
}

__global__ void k_min_edge(int64_t T, int64_t N, const int32_t *__restrict__ tri, const double *__restrict__ xyz,
                           double *__restrict__ out) {
    __shared__ double red[256];
    double mn = INFINITY;
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < T; k += (int64_t)gridDim.x * blockDim.x) {
        int v[3] = {tri[k], tri[T + k], tri[2 * T + k]};
        for (int e = 0; e < 3; ++e) {
            int a = v[e], b = v[(e + 1) % 3];
            double dx = xyz[a] - xyz[b], dy = xyz[N + a] - xyz[N + b], dz = xyz[2 * N + a] - xyz[2 * N + b];
            mn = fmin(mn, sqrt(dx * dx + dy * dy + dz * dz));
        }
    }
    red[threadIdx.x] = mn;
    __syncthreads();
    for (int s = blockDim.x / 2; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] = fmin(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) out[blockIdx.x] = red[0];
}

int grid_for(int64_t n) { return (int)std::min<int64_t>(div_up(n, 256), 152 * 16); }

void apply_filter(Context &c, StepState &s, const double *X, double *Y) {
    if (s.Pf == 0) {
        if (X != Y) BEM_CUDA(cudaMemcpyAsync(Y, X, 4 * c.N * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
        return;
    }
    if (c.prm.precision == BEM_PREC_FP64) {
        k_filter_apply<<<(unsigned)c.M, 256, (size_t)s.Pf * 4 * sizeof(double), c.stream>>>(
            c.N, s.voff.p, s.filt.shape_of.p, s.filt.g_off.p, s.Pf, s.filt.G.p, s.filt.Gp.p, X, Y);
    } else {  // compensated FP32 on the (hi, lo) copies of G and G+
        const size_t sm = ((size_t)4 * FD_CHUNK + (size_t)s.Pf * 4) * sizeof(float2);
        k_filter_apply_df<<<(unsigned)c.M, FD_THREADS, sm, c.stream>>>(c.N, s.voff.p, s.filt.shape_of.p,
                                                                        s.filt.g_off.p, s.Pf, s.filt.Gs.p,
                                                                        s.filt.Gps.p, X, Y);
    }
    BEM_LAUNCH_CHECK();
}

// out = sum_{j < n} w[j] a[j][.]
struct GuessTerms {
    double w[kQh];
    const double *a[kQh];
    int n;
};
__global__ void k_combine(int64_t N, GuessTerms cb, double *__restrict__ out) {
    int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (i >= N) return;
    double v = cb.w[0] * cb.a[0][i];
    for (int j = 1; j < cb.n; ++j) v += cb.w[j] * cb.a[j][i];
    out[i] = v;
}

// s.q <- the Lagrange polynomial in t through the recorded step-start solutions (degree
// min(guess, recorded - 1)), evaluated at t; unchanged below degree 1
void extrapolate_guess(Context &c, StepState &s, double t) {
    const int k = std::min(s.sp.guess, s.qh_n - 1);
    if (k < 1) return;
    GuessTerms cb{};
    cb.n = k + 1;
    for (int j = 0; j <= k; ++j) {
        const double tj = s.qh_time[s.qh_order[j]];
        double v = 1.0;
        for (int m = 0; m <= k; ++m)
            if (m != j) {
                const double tm = s.qh_time[s.qh_order[m]];
                v *= (t - tm) / (tj - tm);
            }
        cb.w[j] = v;
        cb.a[j] = s.qh.p + (size_t)s.qh_order[j] * c.N;
    }
    k_combine<<<div_up(c.N, 256), 256, 0, c.stream>>>(c.N, cb, s.q.p);
    BEM_LAUNCH_CHECK();
}

// record s.q as the solution at step-start time t (the oldest of kQh is dropped)
void record_start_solution(Context &c, StepState &s, double t) {
    s.qh.resize(kQh * (size_t)c.N);
    const int last = s.qh_order[kQh - 1];
    for (int j = kQh - 1; j > 0; --j) s.qh_order[j] = s.qh_order[j - 1];
    s.qh_order[0] = last;
    s.qh_time[last] = t;
    BEM_CUDA(cudaMemcpyAsync(s.qh.p + (size_t)last * c.N, s.q.p, c.N * sizeof(double), cudaMemcpyDeviceToDevice,
                             c.stream));
    s.qh_n = std::min(kQh, s.qh_n + 1);
}

// f = filtered right-hand side at state y (both [4N]), time t. Updates s.q.
// start: the evaluation at the start of a step (the state y_n at t_n), whose solution is
// recorded; extrap: that solve starts from the extrapolated guess. Runge-Kutta steps do not
// extrapolate: their previous solve (k4) is already at the new step's time.
void rhs(Context &c, StepState &s, const double *y, double t, double *f, bem_step_stats &st, bool start,
         bool extrap) {
    const int64_t N = c.N;
    apply_filter(c, s, y, s.yf.p);
    BEM_CUDA(cudaMemcpyAsync(c.xyz.p, s.yf.p, 3 * N * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
    build_all(c);
    st.mvps += 1;  // the 4-RHS diagonal product
    int it = 0;
    double rr = 0.0;
    const double *phi_hat = s.yf.p + 3 * N;
    auto solve_from = [&](double *q, int &iters, double &relres, double &res0) {
        try {
            solve_internal(c, phi_hat, q, &iters, &relres);
        } catch (const Error &e) {
            if (e.code != BEM_ERR_NOCONV) throw;
            st.nonconverged += 1;
            iters = c.stats.last_iters;
            relres = c.stats.last_relres;
        }
        res0 = c.res_hist.empty() ? 0.0 : c.res_hist.front();
    };
    const bool learned = mlp_active(c);
    // the base start of a step-start solve: the extrapolated guess (guess >= 1) or the previous q;
    // the learned guess, when active, predicts its correction
    if (start && extrap) extrapolate_guess(c, s, t);
    if (learned) {
        // samples and guesses only in the Adams-Bashforth phase (one solve per step)
        // samples and guesses at the Adams-Bashforth step starts only (one per step)
        mlp_before_solve(c, phi_hat, s.q.p, start && extrap);  // with the network in use, s.q becomes its guess
        if (mlp_compare(c)) {                 // the same solve from the fallback q_prev, for the record
            s.ytmp.resize(4 * N);
            DevBuf<double> qf;
            qf.resize(N);
            BEM_CUDA(cudaMemcpyAsync(qf.p, mlp_qprev(c), N * sizeof(double), cudaMemcpyDeviceToDevice, c.stream));
            int itf = 0;
            double rrf = 0.0, r0f = 0.0;
            solve_from(qf.p, itf, rrf, r0f);
            MlpStats &ms = mlp_stats(c);
            ms.iters_fallback += itf;
            ms.res0_fallback += r0f;
            st.mvps += c.stats.last_mvps + 1;
        }
    }
    double res0 = 0.0;
    solve_from(s.q.p, it, rr, res0);
    if (start) record_start_solution(c, s, t);
    if (learned) {
        mlp_after_solve(c, s.q.p);
        if (mlp_compare(c)) {
            MlpStats &ms = mlp_stats(c);
            ms.solves += 1;
            ms.iters_guess += it;
            ms.res0_guess += res0;
        }
    }
    st.gmres_iters += it;
    st.mvps += c.stats.last_mvps + 1;  // GMRES products plus the right-hand side
    st.max_relres = std::max(st.max_relres, rr);
    st.rhs_calls += 1;
    PhaseScope ps(c, PH_GEOMETRY);
    const int tb = 256;
    s.vt.resize(3 * N);
    s.H.resize(N);
    c.tri_tmp.resize(2 * (size_t)c.T);
    if (c.T > 0) {
        k_tri_nxv<<<div_up(c.T, tb), tb, 0, c.stream>>>(c.T, N, s.yf.p, s.yf.p + 3 * N, c.tri.p, c.tri_tmp.p);
        BEM_LAUNCH_CHECK();
    }
    k_tangential<<<div_up(N, tb), tb, 0, c.stream>>>(N, c.tri_tmp.p, c.v2t_off.p, c.v2t.p, c.s.p, c.nrm.p, s.vt.p);
    BEM_LAUNCH_CHECK();
    DevBuf<int> &bad = c.chk[3];
    bad.resize(1);
    BEM_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), c.stream));
    k_curvature<<<div_up(N, tb), tb, 0, c.stream>>>(N, s.yf.p, c.nrm.p, s.nbr5.p, s.H.p, bad.p);
    BEM_LAUNCH_CHECK();
    k_volumes<<<(unsigned)c.M, 256, 0, c.stream>>>(N, c.T, s.toff.p, c.tri.p, s.yf.p, s.V.p);
    BEM_LAUNCH_CHECK();
    k_pressure<<<div_up(c.M, tb), tb, 0, c.stream>>>((int)c.M, s.V.p, s.V0.p, s.a0.p, s.sp.sigma, s.sp.kappa, s.pg.p);
    BEM_LAUNCH_CHECK();
    double F = 1.0 - s.sp.pa * sin(s.sp.omega * t);
    k_assemble<<<div_up(N, tb), tb, 0, c.stream>>>(N, s.q.p, c.nrm.p, s.vt.p, s.H.p, s.pg.p, s.bub_of.p, s.sp.sigma,
                                                    F, f);
    BEM_LAUNCH_CHECK();
    apply_filter(c, s, f, f);
    int hb = 0;
    BEM_CUDA(cudaMemcpyAsync(&hb, bad.p, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    BEM_CUDA(cudaStreamSynchronize(c.stream));
    if (hb) fail(BEM_ERR_MESH, "degenerate five-neighbour curvature fit");
}

}  // namespace

// One least-squares spherical-harmonic basis (degrees 0..pf-1) per distinct initial bubble
// shape: bubbles whose unit directions from their centroid coincide share G and G+.
void find_shapes(const Context &c, const std::vector<double> &hx, std::vector<BubbleShape> &shapes,
                 std::vector<int32_t> &shape_of) {
    const int64_t N = c.N, M = c.M;
    shapes.clear();
    shape_of.assign(M, 0);
    auto dir = [&](int64_t j, double cx, double cy, double cz, double *d) {
        d[0] = hx[j] - cx;
        d[1] = hx[N + j] - cy;
        d[2] = hx[2 * N + j] - cz;
        double l = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
        for (int k = 0; k < 3; ++k) d[k] /= l;
    };
    for (int64_t m = 0; m < M; ++m) {
        int64_t a = c.vert_off[m], b = c.vert_off[m + 1];
        int nd = (int)(b - a);
        double cx = 0, cy = 0, cz = 0;
        for (int64_t j = a; j < b; ++j) {
            cx += hx[j];
            cy += hx[N + j];
            cz += hx[2 * N + j];
        }
        cx /= nd;
        cy /= nd;
        cz /= nd;
        int found = -1;
        for (size_t k = 0; k < shapes.size() && found < 0; ++k) {
            const BubbleShape &sh = shapes[k];
            if (sh.nd != nd) continue;
            int64_t ra = c.vert_off[sh.rep];
            bool same = true;
            for (int i = 0; i < nd && same; ++i) {
                double d1[3], d2[3];
                dir(a + i, cx, cy, cz, d1);
                dir(ra + i, sh.cx, sh.cy, sh.cz, d2);
                for (int k2 = 0; k2 < 3; ++k2) same &= std::fabs(d1[k2] - d2[k2]) < 1e-9;
            }
            if (same) found = (int)k;
        }
        if (found < 0) {
            shapes.push_back({m, nd, cx, cy, cz});
            found = (int)shapes.size() - 1;
        }
        shape_of[m] = found;
    }
}

// Eigenvector of the smallest eigenvalue of a symmetric 3x3 matrix (cyclic Jacobi rotations).
static void smallest_eigvec3(double A[3][3], double out[3]) {
    double V[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};
    for (int sweep = 0; sweep < 50; ++sweep) {
        const double off = A[0][1] * A[0][1] + A[0][2] * A[0][2] + A[1][2] * A[1][2];
        if (off < 1e-30 * (A[0][0] * A[0][0] + A[1][1] * A[1][1] + A[2][2] * A[2][2] + 1e-300)) break;
        for (int p = 0; p < 2; ++p)
            for (int q = p + 1; q < 3; ++q) {
                if (A[p][q] == 0.0) continue;
                const double th = 0.5 * (A[q][q] - A[p][p]) / A[p][q];
                const double t = (th >= 0 ? 1.0 : -1.0) / (std::fabs(th) + std::sqrt(th * th + 1.0));
                const double cs = 1.0 / std::sqrt(t * t + 1.0), sn = t * cs;
                for (int k = 0; k < 3; ++k) {  // A <- A J
                    const double akp = A[k][p], akq = A[k][q];
                    A[k][p] = cs * akp - sn * akq;
                    A[k][q] = sn * akp + cs * akq;
                }
                for (int k = 0; k < 3; ++k) {  // A <- J^T A
                    const double apk = A[p][k], aqk = A[q][k];
                    A[p][k] = cs * apk - sn * aqk;
                    A[q][k] = sn * apk + cs * aqk;
                }
                for (int k = 0; k < 3; ++k) {
                    const double vkp = V[k][p], vkq = V[k][q];
                    V[k][p] = cs * vkp - sn * vkq;
                    V[k][q] = sn * vkp + cs * vkq;
                }
            }
    }
    int m = 0;
    for (int k = 1; k < 3; ++k)
        if (A[k][k] < A[m][m]) m = k;
    for (int k = 0; k < 3; ++k) out[k] = V[k][m];
}

// Rows of the toroidal filter's basis (Section 3.6, Eq. (spherical7), in real form) for the nd
// points of a ring-shaped bubble starting at vertex v0 of the host coordinates hx [3][N]: the
// axis is the direction of least second moment about the centroid, phi the angle about it,
// theta the angle about the centre circle (radius: the mean distance from the axis); columns 1
// and cos / sin(n theta + m phi) for |n|, |m| <= h with n > 0, or n = 0 and m > 0.
static void torus_rows(const std::vector<double> &hx, int64_t N, int64_t v0, int nd, int h, int ld,
                       std::vector<double> &G) {
    double c[3] = {0, 0, 0};
    for (int i = 0; i < nd; ++i)
        for (int d = 0; d < 3; ++d) c[d] += hx[d * N + v0 + i];
    for (double &v : c) v /= nd;
    double S[3][3] = {{0}};
    for (int i = 0; i < nd; ++i) {
        double d[3];
        for (int k = 0; k < 3; ++k) d[k] = hx[k * N + v0 + i] - c[k];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) S[a][b] += d[a] * d[b];
    }
    double ax[3];
    smallest_eigvec3(S, ax);
    // e1: the coordinate axis least aligned with the ring axis, projected; e2 = ax x e1
    int m0 = 0;
    for (int k = 1; k < 3; ++k)
        if (std::fabs(ax[k]) < std::fabs(ax[m0])) m0 = k;
    double e1[3] = {0, 0, 0};
    e1[m0] = 1.0;
    const double dp = e1[0] * ax[0] + e1[1] * ax[1] + e1[2] * ax[2];
    double n1 = 0.0;
    for (int k = 0; k < 3; ++k) {
        e1[k] -= dp * ax[k];
        n1 += e1[k] * e1[k];
    }
    for (double &v : e1) v /= std::sqrt(n1);
    const double e2[3] = {ax[1] * e1[2] - ax[2] * e1[1], ax[2] * e1[0] - ax[0] * e1[2], ax[0] * e1[1] - ax[1] * e1[0]};
    std::vector<double> fphi(nd), rho(nd), z(nd);
    double rmean = 0.0;
    for (int i = 0; i < nd; ++i) {
        double d[3];
        for (int k = 0; k < 3; ++k) d[k] = hx[k * N + v0 + i] - c[k];
        const double u = d[0] * e1[0] + d[1] * e1[1] + d[2] * e1[2];
        const double v = d[0] * e2[0] + d[1] * e2[1] + d[2] * e2[2];
        z[i] = d[0] * ax[0] + d[1] * ax[1] + d[2] * ax[2];
        fphi[i] = std::atan2(v, u);
        rho[i] = std::hypot(u, v);
        rmean += rho[i];
    }
    rmean /= nd;
    G.assign((size_t)nd * ld, 0.0);
    for (int i = 0; i < nd; ++i) {
        const double th = std::atan2(z[i], rho[i] - rmean);
        double *row = G.data() + (size_t)i * ld;
        int col = 0;
        row[col++] = 1.0;
        for (int n = 0; n <= h; ++n)
            for (int m = -h; m <= h; ++m) {
                if (n == 0 && m <= 0) continue;
                const double arg = n * th + m * fphi[i];
                row[col++] = std::cos(arg);
                row[col++] = std::sin(arg);
            }
    }
}

// One least-squares basis per distinct initial bubble shape (bubbles whose unit directions from
// their centroid coincide share it): the real spherical harmonics of degrees 0..pf-1 (pf^2
// columns) for sphere-like bubbles (Euler characteristic 2), the real 2D Fourier basis of the
// torus angles with |n|, |m| <= pf/2 ((2 floor(pf/2) + 1)^2 columns) for ring-like bubbles
// (Euler characteristic 0) when allow_torus is set. Every shape's G is stored with B.Pf
// columns, the largest count, zero-padded (a zero column adds nothing to the projection).
void build_sh_basis(Context &c, int pf, ShBasis &B, int *bad, const double *xyz, bool allow_torus) {
    const int64_t N = c.N, M = c.M;
    cudaStream_t st = c.stream;
    if (!xyz) xyz = c.xyz.p;
    B.pf = pf;
    B.Pf = pf * pf;
    if (pf > 0) {
        std::vector<double> hx(3 * N);
        BEM_CUDA(cudaMemcpyAsync(hx.data(), xyz, 3 * N * sizeof(double), cudaMemcpyDeviceToHost, st));
        BEM_CUDA(cudaStreamSynchronize(st));
        std::vector<BubbleShape> shapes;
        std::vector<int32_t> shape_of;
        find_shapes(c, hx, shapes, shape_of);
        const int h = pf / 2, Ptor = (2 * h + 1) * (2 * h + 1);
        std::vector<int> kind(shapes.size(), 0), Pk(shapes.size(), pf * pf);  // 0 sphere, 1 torus
        for (size_t k = 0; k < shapes.size(); ++k) {
            const int64_t r = shapes[k].rep;
            const int64_t chi = (int64_t)shapes[k].nd - (c.tri_off[r + 1] - c.tri_off[r]) / 2;
            if (chi == 0 && allow_torus) {
                kind[k] = 1;
                Pk[k] = Ptor;
            } else if (chi != 2) {
                fail(BEM_ERR_MESH, "shape filter: bubble " + std::to_string(r) + " is neither sphere- nor ring-like " +
                                       "(Euler characteristic " + std::to_string(chi) + ")");
            }
        }
        B.Pf = *std::max_element(Pk.begin(), Pk.end());
        for (size_t k = 0; k < shapes.size(); ++k)
            if (shapes[k].nd < Pk[k]) fail(BEM_ERR_MESH, "bubble with fewer vertices than filter coefficients");
        std::vector<int64_t> goff(shapes.size() + 1, 0);
        for (size_t k = 0; k < shapes.size(); ++k) goff[k + 1] = goff[k] + (int64_t)shapes[k].nd * B.Pf;
        B.G.resize(goff.back());
        B.Gp.resize(goff.back());
        BEM_CUDA(cudaMemsetAsync(B.G.p, 0, goff.back() * sizeof(double), st));
        DevBuf<double> scratch, A;
        int ndmax = 0;
        for (auto &sh : shapes) ndmax = std::max(ndmax, sh.nd);
        scratch.resize((size_t)ndmax * pf * pf);
        A.resize((size_t)B.Pf * B.Pf);
        std::vector<double> Gt;
        for (size_t k = 0; k < shapes.size(); ++k) {
            const BubbleShape &sh = shapes[k];
            if (kind[k] == 0) {
                k_filter_G<<<div_up(sh.nd, 128), 128, 0, st>>>(sh.nd, xyz, N, c.vert_off[sh.rep], sh.cx, sh.cy, sh.cz,
                                                               pf, B.Pf, B.G.p + goff[k], scratch.p);
                BEM_LAUNCH_CHECK();
            } else {
                torus_rows(hx, N, c.vert_off[sh.rep], sh.nd, h, B.Pf, Gt);
                BEM_CUDA(cudaMemcpyAsync(B.G.p + goff[k], Gt.data(), Gt.size() * sizeof(double), cudaMemcpyHostToDevice,
                                         st));
                BEM_CUDA(cudaStreamSynchronize(st));  // Gt is reused
            }
            k_filter_pinv<<<1, 256, 0, st>>>(sh.nd, Pk[k], B.Pf, B.G.p + goff[k], A.p, B.Gp.p + goff[k], bad);
            BEM_LAUNCH_CHECK();
        }
        B.Gs.resize(goff.back());
        B.Gps.resize(goff.back());
        for (size_t k = 0; k < shapes.size(); ++k) {
            const int64_t n = goff[k + 1] - goff[k];
            k_split_df<<<grid_for(n), 256, 0, st>>>(shapes[k].nd, B.Pf, true, B.G.p + goff[k], B.Gs.p + goff[k]);
            k_split_df<<<grid_for(n), 256, 0, st>>>(shapes[k].nd, B.Pf, false, B.Gp.p + goff[k], B.Gps.p + goff[k]);
            BEM_LAUNCH_CHECK();
        }
        B.shape_of.resize(M);
        B.g_off.resize(shapes.size());
        BEM_CUDA(cudaMemcpyAsync(B.shape_of.p, shape_of.data(), M * sizeof(int32_t), cudaMemcpyHostToDevice, st));
        BEM_CUDA(cudaMemcpyAsync(B.g_off.p, goff.data(), shapes.size() * sizeof(int64_t), cudaMemcpyHostToDevice, st));
        BEM_CUDA(cudaStreamSynchronize(st));
    }
}

void step_init(Context &c, const double *phi0_dev, const double *q0_dev, const bem_step_params &sp) {
    if (!c.mesh_ok) fail(BEM_ERR_NOT_BUILT, "no mesh uploaded");
    if (sp.pf < 0 || sp.pf > 11) fail(BEM_ERR_ARG, "pf must be in 0..11");
    if (sp.guess < 0 || sp.guess > kGuessMax) fail(BEM_ERR_ARG, "guess must be in 0..3");
    if (sp.ab_order < 1 || sp.ab_order > 6) fail(BEM_ERR_ARG, "ab_order must be in 1..6");
    if (sp.corrector != 0 && (sp.corrector != 1 || sp.ab_order < 4))
        fail(BEM_ERR_ARG, "corrector must be 0, or 1 with ab_order 4..6");
    if (sp.rk_order < 4 || sp.rk_order > 6) fail(BEM_ERR_ARG, "rk_order must be 4, 5 or 6");
    if (!(sp.pa > 0.0) && !(sp.dt > 0.0)) fail(BEM_ERR_ARG, "pa must be > 0 unless dt is given");
    StepState &s = state_of(c);
    const int64_t N = c.N, M = c.M;
    cudaStream_t st = c.stream;
    const int tb = 256;
    s.sp = sp;
    s.t = 0.0;
    s.steps = 0;
    s.nhist = 0;
    s.qh_n = 0;
    for (int i = 0; i < 5; ++i) s.order[i] = i;
    for (auto *b : {&s.y, &s.ytmp, &s.yf, &s.f}) b->resize(4 * N);
    const int nstages = kRK[sp.rk_order - 4].s;
    for (int i = 0; i < nstages; ++i) s.ks[i].resize(4 * N);
    if (sp.corrector) s.fp.resize(4 * N);
    s.hist.resize(5 * 4 * N);
    s.q.resize(N);
    if (q0_dev) BEM_CUDA(cudaMemcpyAsync(s.q.p, q0_dev, N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    else BEM_CUDA(cudaMemsetAsync(s.q.p, 0, N * sizeof(double), st));
    BEM_CUDA(cudaMemcpyAsync(s.y.p, c.xyz.p, 3 * N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    s.x0.resize(3 * N);
    BEM_CUDA(cudaMemcpyAsync(s.x0.p, c.xyz.p, 3 * N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    BEM_CUDA(cudaMemcpyAsync(s.y.p + 3 * N, phi0_dev, N * sizeof(double), cudaMemcpyDeviceToDevice, st));
    s.voff.resize(M + 1);
    s.toff.resize(M + 1);
    BEM_CUDA(cudaMemcpyAsync(s.voff.p, c.vert_off.data(), (M + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    BEM_CUDA(cudaMemcpyAsync(s.toff.p, c.tri_off.data(), (M + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    s.bub_of.resize(N);
    k_bubble_of<<<(unsigned)M, 256, 0, st>>>((int)M, s.voff.p, s.bub_of.p);
    BEM_LAUNCH_CHECK();
    // five-neighbour lists
    DevBuf<int> bad;
    bad.resize(1);
    BEM_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
    s.nbr5.resize(5 * N);
    k_nbr5<<<div_up(N, tb), tb, 0, st>>>(N, c.T, c.tri.p, c.v2t_off.p, c.v2t.p, s.nbr5.p, bad.p);
    BEM_LAUNCH_CHECK();
    // V_m0, a_m0 of the initial mesh
    s.V.resize(M);
    s.V0.resize(M);
    s.a0.resize(M);
    s.pg.resize(M);
    k_volumes<<<(unsigned)M, 256, 0, st>>>(N, c.T, s.toff.p, c.tri.p, c.xyz.p, s.V.p);
    BEM_LAUNCH_CHECK();
    k_init_bubbles<<<div_up(M, tb), tb, 0, st>>>((int)M, s.V.p, s.V0.p, s.a0.p);
    BEM_LAUNCH_CHECK();
    // step size, Eq. (3.12)
    if (sp.dt > 0.0) {
        s.dt = sp.dt;
    } else {
        int nb = std::min<int64_t>(div_up(c.T, tb), 1024);
        DevBuf<double> part;
        part.resize(nb);
        k_min_edge<<<nb, tb, 0, st>>>(c.T, N, c.tri.p, c.xyz.p, part.p);
        BEM_LAUNCH_CHECK();
        std::vector<double> h(nb);
        BEM_CUDA(cudaMemcpyAsync(h.data(), part.p, nb * sizeof(double), cudaMemcpyDeviceToHost, st));
        BEM_CUDA(cudaStreamSynchronize(st));
        double mn = *std::min_element(h.begin(), h.end());
        s.dt = sp.courant * mn / std::sqrt(sp.pa);
    }
    // shape filters: one per distinct set of unit directions from the bubble centroid
    build_sh_basis(c, sp.pf, s.filt, bad.p, nullptr, true);
    s.Pf = s.filt.Pf;
    int hb = 0;
    BEM_CUDA(cudaMemcpyAsync(&hb, bad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    BEM_CUDA(cudaStreamSynchronize(st));
    if (hb & 1) fail(BEM_ERR_MESH, "vertex with fewer than five neighbours");
    if (hb & 4) fail(BEM_ERR_MESH, "singular shape-filter normal matrix");
    s.ready = true;
}

void step_advance(Context &c, bem_step_stats &st) {
    StepState &s = state_of(c);
    if (!s.ready) fail(BEM_ERR_NOT_BUILT, "bem_step_init has not been called");
    const int64_t n4 = 4 * c.N;
    const double dt = s.dt, t = s.t;
    cudaStream_t str = c.stream;
    const int g = grid_for(n4);
    const int order = s.sp.ab_order;
    std::memset(&st, 0, sizeof(st));
    auto slot = [&](int i) { return s.hist.p + (size_t)s.order[i] * n4; };
    // push f (the right-hand side at the step start) to the history, newest first
    auto push = [&](const double *f) {
        const int last = s.order[4];
        for (int i = 4; i > 0; --i) s.order[i] = s.order[i - 1];
        s.order[0] = last;
        BEM_CUDA(cudaMemcpyAsync(slot(0), f, n4 * sizeof(double), cudaMemcpyDeviceToDevice, str));
        s.nhist = std::min(5, s.nhist + 1);
    };
    auto lincomb = [&](const double *y, double h, const LinTerms &lt, double *out) {
        k_lincomb<<<g, 256, 0, str>>>(n4, h, y, lt, out);
        BEM_LAUNCH_CHECK();
    };
    if (s.nhist < order - 1) {
        // Runge-Kutta start: stage i at t + c_i dt from y + dt sum_j a_ij k_j
        const Tableau &tb = kRK[s.sp.rk_order - 4];
        for (int i = 0; i < tb.s; ++i) {
            const double *yi = s.y.p;
            if (i > 0) {
                LinTerms lt{};
                for (int j = 0; j < i; ++j)
                    if (tb.a[i][j] != 0.0) {
                        lt.f[lt.n] = s.ks[j].p;
                        lt.w[lt.n] = tb.a[i][j];
                        ++lt.n;
                    }
                lincomb(s.y.p, dt, lt, s.ytmp.p);
                yi = s.ytmp.p;
            }
            rhs(c, s, yi, t + tb.c[i] * dt, s.ks[i].p, st, i == 0, false);
        }
        push(s.ks[0].p);
        LinTerms lt{};
        for (int i = 0; i < tb.s; ++i)
            if (tb.b[i] != 0.0) {
                lt.f[lt.n] = s.ks[i].p;
                lt.w[lt.n] = tb.b[i];
                ++lt.n;
            }
        lincomb(s.y.p, dt, lt, s.y.p);
    } else {
        // Adams-Bashforth of the given order from f_n and the history
        rhs(c, s, s.y.p, t, s.f.p, st, true, true);
        LinTerms lt{};
        lt.n = order;
        lt.f[0] = s.f.p;
        lt.w[0] = kAB[order - 1][0];
        for (int j = 1; j < order; ++j) {
            lt.f[j] = slot(j - 1);
            lt.w[j] = kAB[order - 1][j];
        }
        if (s.sp.corrector) {
            // predict, evaluate at t + dt, correct (Adams-Moulton of the same order)
            lincomb(s.y.p, dt, lt, s.ytmp.p);
            rhs(c, s, s.ytmp.p, t + dt, s.fp.p, st, false, false);
            LinTerms lc{};
            lc.n = order;
            lc.f[0] = s.fp.p;
            lc.w[0] = kAM[order - 4][0];
            lc.f[1] = s.f.p;
            lc.w[1] = kAM[order - 4][1];
            for (int j = 2; j < order; ++j) {
                lc.f[j] = slot(j - 2);
                lc.w[j] = kAM[order - 4][j];
            }
            lincomb(s.y.p, dt, lc, s.y.p);
        } else {
            lincomb(s.y.p, dt, lt, s.y.p);
        }
        push(s.f.p);
    }
    s.t = t + dt;
    s.steps += 1;
    st.t = s.t;
    st.dt = dt;
    st.steps = s.steps;
    s.last = st;
    BEM_CUDA(cudaStreamSynchronize(str));
}

void step_get_state(Context &c, double *xyz, double *phi, double *q, double *t) {
    StepState &s = state_of(c);
    if (!s.ready) fail(BEM_ERR_NOT_BUILT, "bem_step_init has not been called");
    const int64_t N = c.N;
    auto cp = [&](double *dst, const double *src, int64_t n) {
        if (!dst) return;
        auto k = is_device_ptr(c, dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        BEM_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double), k, c.stream));
    };
    cp(xyz, s.y.p, 3 * N);
    cp(phi, s.y.p + 3 * N, N);
    cp(q, s.q.p, N);
    BEM_CUDA(cudaStreamSynchronize(c.stream));
    if (t) *t = s.t;
}

void step_filter(Context &c, const double *x, double *y) {
    StepState &s = state_of(c);
    if (!s.ready) fail(BEM_ERR_NOT_BUILT, "bem_step_init has not been called");
    if (!x || !y) fail(BEM_ERR_ARG, "null x or y");
    const int64_t n4 = 4 * c.N;
    const bool hx = !is_device_ptr(c, x), hy = !is_device_ptr(c, y);
    if (hx || hy) s.fio.resize(n4);
    const double *src = x;
    if (hx) {
        BEM_CUDA(cudaMemcpyAsync(s.fio.p, x, n4 * sizeof(double), cudaMemcpyHostToDevice, c.stream));
        src = s.fio.p;
    }
    double *dst = hy ? s.fio.p : y;
    apply_filter(c, s, src, dst);  // in place when both are the staging buffer
    if (hy) BEM_CUDA(cudaMemcpyAsync(y, dst, n4 * sizeof(double), cudaMemcpyDeviceToHost, c.stream));
    BEM_CUDA(cudaStreamSynchronize(c.stream));
}

// ------------------------------------------------------------------------------ checkpoint
// Layout of a checkpoint: this header, then FP64 arrays r(0) [3N], y = (r, phi) [4N], q [N],
// the right-hand-side history [5][4N] (slots in storage order; `order` says which is newest)
// and the step-start solutions of the extrapolated guess [kQh][N].
struct CkptHeader {
    char magic[8];
    int32_t version, tuned_level, tuned_stages, tuned_p2p_blocks, tuned_overlap, reserved;
    int64_t N, T, M;
    bem_step_params sp;
    double t, dt;
    int64_t steps;
    int32_t nhist, order[5];
    int32_t qh_n, qh_order[kQh];
    double qh_time[kQh];
};
constexpr char kCkptMagic[8] = {'B', 'E', 'M', 'S', 'T', 'E', 'P', '1'};

int64_t step_checkpoint_size(const Context &c) {
    return (int64_t)sizeof(CkptHeader) + (int64_t)(3 + 4 + 1 + 5 * 4 + kQh) * c.N * (int64_t)sizeof(double);
}

void step_save(Context &c, void *buf, int64_t cap) {
    StepState &s = state_of(c);
    if (!s.ready) fail(BEM_ERR_NOT_BUILT, "bem_step_init has not been called");
    const int64_t N = c.N, need = step_checkpoint_size(c);
    if (cap < need) fail(BEM_ERR_ARG, "checkpoint buffer too small: " + std::to_string(cap) + " < " + std::to_string(need));
    CkptHeader h{};
    std::memcpy(h.magic, kCkptMagic, 8);
    h.version = 1;
    h.tuned_level = c.tuned_level;
    h.tuned_stages = c.tuned_stages;
    h.tuned_p2p_blocks = c.tuned_p2p_blocks;
    h.tuned_overlap = c.tuned_overlap;
    h.N = N;
    h.T = c.T;
    h.M = c.M;
    h.sp = s.sp;
    h.t = s.t;
    h.dt = s.dt;
    h.steps = s.steps;
    h.nhist = s.nhist;
    for (int i = 0; i < 5; ++i) h.order[i] = s.order[i];
    h.qh_n = s.qh_n;
    for (int i = 0; i < kQh; ++i) {
        h.qh_order[i] = s.qh_order[i];
        h.qh_time[i] = s.qh_time[i];
    }
    s.qh.resize((size_t)kQh * N);  // allocated at the first recorded solve; zeros before
    if (s.qh_n == 0) BEM_CUDA(cudaMemsetAsync(s.qh.p, 0, (size_t)kQh * N * sizeof(double), c.stream));
    unsigned char *o = static_cast<unsigned char *>(buf);
    BEM_CUDA(cudaMemcpyAsync(o, &h, sizeof(h), cudaMemcpyDefault, c.stream));
    int64_t off = sizeof(h);
    auto put = [&](const double *src, int64_t n) {
        BEM_CUDA(cudaMemcpyAsync(o + off, src, n * sizeof(double), cudaMemcpyDefault, c.stream));
        off += n * (int64_t)sizeof(double);
    };
    put(s.x0.p, 3 * N);
    put(s.y.p, 4 * N);
    put(s.q.p, N);
    put(s.hist.p, 5 * 4 * N);
    put(s.qh.p, kQh * N);
    BEM_CUDA(cudaStreamSynchronize(c.stream));
}

void step_load(Context &c, const void *buf, int64_t size) {
    if (!c.mesh_ok || c.points_only) fail(BEM_ERR_NOT_BUILT, "upload the mesh (same connectivity) first");
    CkptHeader h{};
    if (size < (int64_t)sizeof(h)) fail(BEM_ERR_ARG, "checkpoint too small");
    BEM_CUDA(cudaMemcpy(&h, buf, sizeof(h), cudaMemcpyDefault));
    if (std::memcmp(h.magic, kCkptMagic, 8) != 0 || h.version != 1) fail(BEM_ERR_ARG, "not a time-step checkpoint");
    if (h.N != c.N || h.T != c.T || h.M != c.M)
        fail(BEM_ERR_ARG, "checkpoint of another mesh (N, T or M differ)");
    const int64_t N = c.N;
    if (size < step_checkpoint_size(c)) fail(BEM_ERR_ARG, "checkpoint truncated");
    const unsigned char *in = static_cast<const unsigned char *>(buf);
    int64_t off = sizeof(h);
    auto at = [&](int64_t n) {
        const double *p = reinterpret_cast<const double *>(in + off);
        off += n * (int64_t)sizeof(double);
        return p;
    };
    const double *x0 = at(3 * N), *y = at(4 * N), *q = at(N), *hist = at(5 * 4 * N), *qh = at(kQh * N);
    // the fixed parts (filters, V0, a0, neighbour lists, dt) are rebuilt from r(0) as
    // bem_step_init builds them; phi0 and q0 are placeholders overwritten below
    BEM_CUDA(cudaMemcpyAsync(c.xyz.p, x0, 3 * N * sizeof(double), cudaMemcpyDefault, c.stream));
    c.built = false;
    c.bp.ready = false;
    DevBuf<double> tmp;
    tmp.resize(2 * N);
    BEM_CUDA(cudaMemcpyAsync(tmp.p, y + 3 * N, N * sizeof(double), cudaMemcpyDefault, c.stream));
    BEM_CUDA(cudaMemcpyAsync(tmp.p + N, q, N * sizeof(double), cudaMemcpyDefault, c.stream));
    step_init(c, tmp.p, tmp.p + N, h.sp);
    StepState &s = state_of(c);
    BEM_CUDA(cudaMemcpyAsync(s.y.p, y, 4 * N * sizeof(double), cudaMemcpyDefault, c.stream));
    BEM_CUDA(cudaMemcpyAsync(s.hist.p, hist, 5 * 4 * N * sizeof(double), cudaMemcpyDefault, c.stream));
    s.qh.resize((size_t)kQh * N);
    BEM_CUDA(cudaMemcpyAsync(s.qh.p, qh, (size_t)kQh * N * sizeof(double), cudaMemcpyDefault, c.stream));
    s.t = h.t;
    s.dt = h.dt;
    s.steps = h.steps;
    s.nhist = h.nhist;
    for (int i = 0; i < 5; ++i) s.order[i] = h.order[i];
    s.qh_n = h.qh_n;
    for (int i = 0; i < kQh; ++i) {
        s.qh_order[i] = h.qh_order[i];
        s.qh_time[i] = h.qh_time[i];
    }
    if (h.tuned_level > 0 && c.prm.leaf_target == 0 && c.prm.fixed_level == 0) {
        // the saved run's autotuned tiles (no new timing run on this mesh)
        c.tuned_level = h.tuned_level;
        c.tuned_stages = h.tuned_stages;
        c.tuned_p2p_blocks = h.tuned_p2p_blocks;
        if (c.prm.overlap < 0) c.tuned_overlap = h.tuned_overlap;
    }
    BEM_CUDA(cudaStreamSynchronize(c.stream));
}

void step_set_state(Context &c, const double *xyz, const double *phi, const double *q) {
    StepState &s = state_of(c);
    if (!s.ready) fail(BEM_ERR_NOT_BUILT, "bem_step_init has not been called");
    const int64_t N = c.N;
    auto cp = [&](double *dst, const double *src, int64_t n) {
        if (!src) return;
        BEM_CUDA(cudaMemcpyAsync(dst, src, n * sizeof(double), cudaMemcpyDefault, c.stream));
    };
    cp(s.y.p, xyz, 3 * N);
    cp(s.y.p + 3 * N, phi, N);
    cp(s.q.p, q, N);
    BEM_CUDA(cudaStreamSynchronize(c.stream));
}

void step_free(StepState *s) { delete s; }

const double *step_initial_xyz(Context &c) {
    StepState &s = state_of(c);
    if (!s.ready) fail(BEM_ERR_NOT_BUILT, "bem_step_init has not been called");
    return s.x0.p;
}

}  // namespace bem
