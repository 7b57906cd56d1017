// Bubble-block preconditioner for the GMRES solve of L q = b (gmres_precond = 2).
//
// The paper solves with unpreconditioned GMRES and mentions a preconditioned flexible GMRES
// as the alternative it tried (Section 3.8). The slow GMRES components here are those of each
// bubble's own single-layer block: on a sphere of radius R its eigenvalues are R/(2n+1), a
// spread that grows with the mesh resolution. This preconditioner removes them: for every
// distinct bubble mesh (same connectivity; every icosphere of one level is one group), it
// inverts the single-layer matrix of the isolated representative bubble, including its
// singular diagonal from the identity of Eq. (s5) summed over that bubble alone, and scales
// it to unit size. Bubble m of the group is
// preconditioned by (1/R_m) times that inverse, R_m its current mean centroid distance (the
// single layer of a bubble scaled by R is R times the unit one). The inverse is built from
// the geometry of the first solve after a mesh upload and kept; only the scales follow the
// bubbles as they move. The solve still stops on the true residual |b - L q| / |b| of the
// unpreconditioned system, so the solution meets the same tolerance.
//
// Setup per shape (n vertices): the n x n block is assembled in FP64 and inverted in place by
// Gauss-Jordan elimination without pivoting (two launches per pivot). The block is K S with K
// the symmetric single-layer kernel matrix and S the diagonal of vertex areas, so every
// leading principal minor is positive when K is positive definite; a pivot that is not
// positive stops the setup with an error. Apply: one GEMM per shape with the bubbles' vertex
// ranges as the right-hand columns: on the tensor cores on the mixed path (both operands split
// into three BF16 pieces, six products accumulated in FP32: as accurate as an FP32 product, so
// the preconditioner stays one fixed linear map, which right-preconditioned GMRES needs), and a
// tiled FP64 GEMM on the FP64 path.
#include "internal.h"
#include "tcgen05.cuh"

#include <cmath>

namespace bem {
namespace {

constexpr double kInv4Pi = 0.0795774715459476678844418816862571810;

// Row i of the isolated bubble's single-layer block (vertices a..a+n-1 in caller order),
// coordinates relative to the centroid c: A_ij = s_j / (4 pi |r_i - r_j|) for j != i and
// A_ii = n_i . [ sum_{j != i} (M_ij r_j - L_ij n_j) + (1/2 + M_ii) r_i ], M_ii = -1/2 - sum M_ij,
// all sums over this bubble only (Eqs. (s3), (s5)).
__global__ void k_bp_assemble(int n, int64_t N, int64_t a, double cx, double cy, double cz,
                              const double *__restrict__ xyz, const double *__restrict__ s,
                              const double *__restrict__ nrm, double *__restrict__ A) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int64_t gi = a + i;
    const double xi = xyz[gi] - cx, yi = xyz[N + gi] - cy, zi = xyz[2 * N + gi] - cz;
    double msum = 0.0, vx = 0.0, vy = 0.0, vz = 0.0;
    for (int j = 0; j < n; ++j) {
        if (j == i) continue;
        const int64_t gj = a + j;
        const double xj = xyz[gj] - cx, yj = xyz[N + gj] - cy, zj = xyz[2 * N + gj] - cz;
        const double dx = xi - xj, dy = yi - yj, dz = zi - zj;
        const double r2 = dx * dx + dy * dy + dz * dz;
        const double rinv = 1.0 / sqrt(r2);
        const double nx = nrm[gj], ny = nrm[N + gj], nz = nrm[2 * N + gj];
        const double lij = s[gj] * kInv4Pi * rinv;
        const double mij = s[gj] * kInv4Pi * (nx * dx + ny * dy + nz * dz) * rinv * rinv * rinv;
        A[(size_t)i * n + j] = lij;
        msum += mij;
        vx += mij * xj - lij * nx;
        vy += mij * yj - lij * ny;
        vz += mij * zj - lij * nz;
    }
    const double mii = -0.5 - msum;
    const double h = 0.5 + mii;
    A[(size_t)i * n + i] = nrm[gi] * (vx + h * xi) + nrm[N + gi] * (vy + h * yi) + nrm[2 * N + gi] * (vz + h * zi);
}

// Gauss-Jordan step k, part 1: A_ij -= A_ik A_kj / A_kk for i != k and j != k (row k and column
// k are read, not written); keeps a copy of the pivot for part 2.
__global__ void k_gj_interior(int n, int k, double *__restrict__ A, double *__restrict__ piv) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    const int i = blockIdx.y;
    const double p = A[(size_t)k * n + k];
    if (i == 0 && j == 0) *piv = p;
    if (i == k || j >= n || j == k) return;
    A[(size_t)i * n + j] -= A[(size_t)i * n + k] * A[(size_t)k * n + j] / p;
}

// Gauss-Jordan step k, part 2: row k /= p, column k = -column k / p, A_kk = 1 / p.
__global__ void k_gj_pivot(int n, int k, double *__restrict__ A, const double *__restrict__ piv,
                           int *__restrict__ bad) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    const double p = *piv;
    if (t == 0 && !(p > 0.0)) atomicOr(bad, 1);
    if (t >= n) return;
    if (t == k) {
        A[(size_t)k * n + k] = 1.0 / p;
    } else {
        A[(size_t)k * n + t] /= p;
        A[(size_t)t * n + k] = -A[(size_t)t * n + k] / p;
    }
}

// inverse at size R -> unit size (times R)
__global__ void k_bp_store(size_t cnt, double R, const double *__restrict__ A, double *__restrict__ o64) {
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < cnt; e += (size_t)gridDim.x * blockDim.x)
        o64[e] = A[e] * R;
}

// per bubble of a shape (one block each): 1 / mean distance of its vertices from their centroid
__global__ void k_bp_scales(int n, int64_t N, const int64_t *__restrict__ voff, const double *__restrict__ xyz,
                            double *__restrict__ scale) {
    __shared__ double red[4][8];
    const int64_t a = voff[blockIdx.x];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    double sx = 0.0, sy = 0.0, sz = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        sx += xyz[a + i];
        sy += xyz[N + a + i];
        sz += xyz[2 * N + a + i];
    }
    for (int o = 16; o > 0; o >>= 1) {
        sx += __shfl_down_sync(0xffffffffu, sx, o);
        sy += __shfl_down_sync(0xffffffffu, sy, o);
        sz += __shfl_down_sync(0xffffffffu, sz, o);
    }
    if (lane == 0) {
        red[0][w] = sx;
        red[1][w] = sy;
        red[2][w] = sz;
    }
    __syncthreads();
    double cx = 0.0, cy = 0.0, cz = 0.0;
    for (int k = 0; k < (int)(blockDim.x >> 5); ++k) {
        cx += red[0][k];
        cy += red[1][k];
        cz += red[2][k];
    }
    cx /= n;
    cy /= n;
    cz /= n;
    double d = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const double dx = xyz[a + i] - cx, dy = xyz[N + a + i] - cy, dz = xyz[2 * N + a + i] - cz;
        d += sqrt(dx * dx + dy * dy + dz * dz);
    }
    for (int o = 16; o > 0; o >>= 1) d += __shfl_down_sync(0xffffffffu, d, o);
    __syncthreads();
    if (lane == 0) red[3][w] = d;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int k = 0; k < (int)(blockDim.x >> 5); ++k) t += red[3][k];
        scale[blockIdx.x] = (double)n / t;
    }
}

// z[voff_b + r] = scale_b * sum_k inv[r][k] y[voff_b + k] for the bubbles b of one shape:
// a 64-row x 32-bubble output tile per block, K in steps of 32 through shared memory.
constexpr int BP_TM = 64, BP_TN = 32, BP_TK = 32, BP_THREADS = 256;

template <class T>
__global__ void __launch_bounds__(BP_THREADS) k_bp_apply(int n, const T *__restrict__ inv, int nb,
                                                         const int64_t *__restrict__ voff,
                                                         const double *__restrict__ scale,
                                                         const double *__restrict__ y, double *__restrict__ z) {
    __shared__ T As[BP_TK][BP_TM + 1];
    __shared__ T Bs[BP_TK][BP_TN + 1];
    __shared__ int64_t sv[BP_TN];
    const int row0 = blockIdx.x * BP_TM, b0 = blockIdx.y * BP_TN;
    const int tid = threadIdx.x, tr = tid & 15, tb = tid >> 4;  // rows tr + 16 i, bubbles 2 tb + j
    if (tid < BP_TN) sv[tid] = (b0 + tid < nb) ? voff[b0 + tid] : -1;
    T acc[4][2];
#pragma unroll
    for (int i = 0; i < 4; ++i) acc[i][0] = acc[i][1] = (T)0;
    for (int k0 = 0; k0 < n; k0 += BP_TK) {
        __syncthreads();
        for (int e = tid; e < BP_TM * BP_TK; e += BP_THREADS) {
            const int r = e / BP_TK, kk = e % BP_TK;
            As[kk][r] = (row0 + r < n && k0 + kk < n) ? inv[(size_t)(row0 + r) * n + k0 + kk] : (T)0;
        }
        for (int e = tid; e < BP_TN * BP_TK; e += BP_THREADS) {
            const int bb = e / BP_TK, kk = e % BP_TK;
            const int64_t v = sv[bb];
            Bs[kk][bb] = (v >= 0 && k0 + kk < n) ? (T)y[v + k0 + kk] : (T)0;
        }
        __syncthreads();
#pragma unroll 8
        for (int kk = 0; kk < BP_TK; ++kk) {
            const T b0v = Bs[kk][2 * tb], b1v = Bs[kk][2 * tb + 1];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                const T av = As[kk][tr + 16 * i];
                acc[i][0] += av * b0v;
                acc[i][1] += av * b1v;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < 2; ++j) {
        const int bb = 2 * tb + j;
        const int64_t v = sv[bb];
        if (v < 0) continue;
        const double sc = scale[b0 + bb];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = row0 + tr + 16 * i;
            if (r < n) z[v + r] = sc * (double)acc[i][j];
        }
    }
}

// Tensor-core form of the block product (mixed precision). For one shape with n vertices and
// nb bubbles, Z (n x nb) = Inv (n x n) Y (n x nb) with D = A B^T on tcgen05: A = Inv (row r is
// K-contiguous), B = Y^T (bubble b's segment is K-contiguous), M = 128 rows, N = 256 bubbles
// per tile, K in steps of 16. Both operands are stored in global memory already in the
// canonical K-major blocks of one K step, [piece][K step][rows][16], so that every stage is
// six contiguous bulk copies (the TMA engine): A from the table split once per build, B from
// the right-hand side split once per application (k_bp_split_y). Thread 0 fills the stages,
// thread 32 issues six MMAs per stage (the small cross terms first) and commits each stage to
// its "empty" barrier; every wait is bounded and raises the error flag when it runs out. The
// epilogue reads the accumulator tile from TMEM (warp w: lanes 32 (w % 4) .. + 31 = rows,
// columns 128 (w / 4) .. + 127 = bubbles) and writes z_b[r] = s_b D[r][b] in FP64, 32
// consecutive rows of one bubble per store instruction.
constexpr int BPC_M = 128, BPC_N = 256, BPC_STAGES = 4, BPC_THREADS = 256;
constexpr uint32_t BPC_A_PIECE = BPC_M * TC_K * 2, BPC_B_PIECE = BPC_N * TC_K * 2;
constexpr uint32_t BPC_STAGE = 3 * (BPC_A_PIECE + BPC_B_PIECE);
constexpr size_t BPC_SMEM = (size_t)BPC_STAGES * BPC_STAGE + 2 * BPC_STAGES * 8 + 16 + 1024;

// Inv (row-major n x n, FP64) -> [3][nks][Mpad x 16] K-major blocks; zero past n.
__global__ void k_bp_split_inv(int n, int nks, int Mpad, const double *__restrict__ inv,
                               __nv_bfloat16 *__restrict__ out) {
    const int64_t units = (int64_t)Mpad * nks * 2;  // (row, 8-wide K chunk)
    const size_t plane = (size_t)nks * Mpad * TC_K;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < units; u += (int64_t)gridDim.x * blockDim.x) {
        const int r = (int)(u / (nks * 2)), k8 = (int)(u % (nks * 2));
        const int ks = k8 >> 1, kk0 = (k8 & 1) * 8;
        __nv_bfloat16 p0[8], p1[8], p2[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int k = ks * TC_K + kk0 + i;
            split3_d(r < n && k < n ? inv[(size_t)r * n + k] : 0.0, p0[i], p1[i], p2[i]);
        }
        const size_t o = (size_t)ks * Mpad * TC_K + kmajor_off(r, kk0);
        *reinterpret_cast<uint4 *>(out + o) = *reinterpret_cast<const uint4 *>(p0);
        *reinterpret_cast<uint4 *>(out + plane + o) = *reinterpret_cast<const uint4 *>(p1);
        *reinterpret_cast<uint4 *>(out + 2 * plane + o) = *reinterpret_cast<const uint4 *>(p2);
    }
}

// y_b (FP64, vertices voff_b .. + n - 1) -> [3][nks][NBpad x 16] K-major blocks; zero past n
// and for the padding bubbles b >= nb. Consecutive threads take consecutive bubbles of one
// 8-wide K chunk, so that a warp's 16-byte pieces form four contiguous 128-byte runs.
__global__ void k_bp_split_y(int n, int nks, int nb, int NBpad, const int64_t *__restrict__ voff,
                             const double *__restrict__ y, __nv_bfloat16 *__restrict__ out) {
    const int64_t units = (int64_t)NBpad * nks * 2;  // (8-wide K chunk, bubble)
    const size_t plane = (size_t)nks * NBpad * TC_K;
    for (int64_t u = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; u < units; u += (int64_t)gridDim.x * blockDim.x) {
        const int b = (int)(u % NBpad), k8 = (int)(u / NBpad);
        const int ks = k8 >> 1, kk0 = (k8 & 1) * 8;
        const double *yb = b < nb ? y + voff[b] : nullptr;
        __nv_bfloat16 p0[8], p1[8], p2[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
            const int k = ks * TC_K + kk0 + i;
            split3_d(yb && k < n ? yb[k] : 0.0, p0[i], p1[i], p2[i]);
        }
        const size_t o = (size_t)ks * NBpad * TC_K + kmajor_off(b, kk0);
        *reinterpret_cast<uint4 *>(out + o) = *reinterpret_cast<const uint4 *>(p0);
        *reinterpret_cast<uint4 *>(out + plane + o) = *reinterpret_cast<const uint4 *>(p1);
        *reinterpret_cast<uint4 *>(out + 2 * plane + o) = *reinterpret_cast<const uint4 *>(p2);
    }
}

__global__ void __launch_bounds__(BPC_THREADS, 1)
    k_bp_apply_tc(int n, int nks, int Mpad, int NBpad, int nb, const __nv_bfloat16 *__restrict__ A,
                  const __nv_bfloat16 *__restrict__ Ys, const int64_t *__restrict__ voff,
                  const double *__restrict__ scale, double *__restrict__ z, int *__restrict__ err) {
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    unsigned char *smem = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + (size_t)BPC_STAGES * BPC_STAGE);
    uint64_t *empty = full + BPC_STAGES;
    uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(empty + BPC_STAGES);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tmem_slot + 1);
    __shared__ int64_t s_v[BPC_N];
    __shared__ double s_sc[BPC_N];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    __shared__ int s_skip;  // one read of the flag, so that the whole block leaves or stays
    if (tid == 0) s_skip = *reinterpret_cast<volatile int *>(err);
    __syncthreads();
    if (s_skip) return;
    const int r0 = blockIdx.x * BPC_M, b0 = blockIdx.y * BPC_N;
    {
        const int b = b0 + tid;  // BPC_THREADS == BPC_N
        s_v[tid] = b < nb ? voff[b] : -1;
        s_sc[tid] = b < nb ? scale[b] : 0.0;
    }
    if (tid == 0) {
        for (int s = 0; s < BPC_STAGES; ++s) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&full[s])));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(&empty[s])));
        }
        *abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                     "n"(BPC_N));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tmem_slot;
    const uint32_t sbase = smem_u32(smem);
    __shared__ int s_last;
    if (tid == 0) {  // producer: six bulk copies per stage
        int issued = -1;
        for (int ks = 0; ks < nks; ++ks) {
            const int st = ks % BPC_STAGES;
            if (ks >= BPC_STAGES &&
                (!mbar_wait(smem_u32(&empty[st]), (uint32_t)((ks / BPC_STAGES - 1) & 1)) || *abort_flag)) {
                *abort_flag = 1;
                break;
            }
            const uint32_t sa = sbase + st * BPC_STAGE, sb = sa + 3 * BPC_A_PIECE, fb = smem_u32(&full[st]);
            mbar_expect_tx(fb, BPC_STAGE);
            for (int piece = 0; piece < 3; ++piece) {
                bulk_g2s(sa + piece * BPC_A_PIECE, A + ((size_t)(piece * nks + ks) * Mpad + r0) * TC_K, BPC_A_PIECE,
                         fb);
                bulk_g2s(sb + piece * BPC_B_PIECE, Ys + ((size_t)(piece * nks + ks) * NBpad + b0) * TC_K,
                         BPC_B_PIECE, fb);
            }
            issued = ks;
        }
        // no copy may still be in flight when the block leaves
        for (int k2 = issued; k2 >= 0 && k2 > issued - BPC_STAGES; --k2)
            if (!mbar_wait(smem_u32(&full[k2 % BPC_STAGES]), (uint32_t)((k2 / BPC_STAGES) & 1))) *abort_flag = 1;
    } else if (tid == 32) {  // MMA issuer
        const uint32_t idesc = make_idesc(BPC_M, BPC_N);
        int ks = 0;
        for (; ks < nks; ++ks) {
            const int st = ks % BPC_STAGES;
            if (!mbar_wait(smem_u32(&full[st]), (uint32_t)((ks / BPC_STAGES) & 1)) || *abort_flag) {
                *abort_flag = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const uint32_t sa = sbase + st * BPC_STAGE, sb = sa + 3 * BPC_A_PIECE;
            const uint32_t a0 = sa, a1 = sa + BPC_A_PIECE, a2 = sa + 2 * BPC_A_PIECE;
            const uint32_t y0 = sb, y1 = sb + BPC_B_PIECE, y2 = sb + 2 * BPC_B_PIECE;
            mma_bf16(tmem, make_desc(a2), make_desc(y0), idesc, ks > 0 ? 1u : 0u);
            mma_bf16(tmem, make_desc(a1), make_desc(y1), idesc, 1u);
            mma_bf16(tmem, make_desc(a0), make_desc(y2), idesc, 1u);
            mma_bf16(tmem, make_desc(a1), make_desc(y0), idesc, 1u);
            mma_bf16(tmem, make_desc(a0), make_desc(y1), idesc, 1u);
            mma_bf16(tmem, make_desc(a0), make_desc(y0), idesc, 1u);
            mma_commit(smem_u32(&empty[st]));
        }
        s_last = ks - 1;
    }
    __syncthreads();
    const int lk = s_last;
    const bool done =
        lk >= 0 && mbar_wait(smem_u32(&empty[lk % BPC_STAGES]), (uint32_t)((lk / BPC_STAGES) & 1));
    const bool ok = !*abort_flag && lk == nks - 1 && done;
    if (!ok && tid == 0) atomicOr(err, 1);
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (ok) {
        const int q4 = warp & 3, half = warp >> 2;
        const int row = r0 + q4 * 32 + lane;
        for (int c0 = half * 128; c0 < half * 128 + 128 && b0 + c0 < nb; c0 += 16) {
            uint32_t v[16];
            const uint32_t taddr = tmem + ((uint32_t)(q4 * 32) << 16) + (uint32_t)c0;
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
                "[%16];"
                : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                  "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
                  "=r"(v[15])
                : "r"(taddr));
            asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
            if (row < n) {
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int64_t vb = s_v[c0 + i];
                    if (vb >= 0) z[vb + row] = s_sc[c0 + i] * (double)__uint_as_float(v[i]);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(BPC_N));
}

// Bubbles whose meshes have the same connectivity (vertex count and triangle list relative to
// their first vertex) share one block inverse: the representative's, scaled by size. A mesh
// copied from one template (every icosphere of one level) is one group however it deforms.
void find_topologies(const Context &c, const std::vector<double> &hx, const std::vector<int32_t> &ht,
                     std::vector<BubbleShape> &shapes, std::vector<int32_t> &shape_of) {
    const int64_t N = c.N, M = c.M, T = c.T;
    shapes.clear();
    shape_of.assign(M, 0);
    for (int64_t m = 0; m < M; ++m) {
        const int64_t a = c.vert_off[m], nd = c.vert_off[m + 1] - a;
        const int64_t ta = c.tri_off[m], nt = c.tri_off[m + 1] - ta;
        int found = -1;
        for (size_t k = 0; k < shapes.size() && found < 0; ++k) {
            const int64_t r = shapes[k].rep;
            const int64_t ra = c.vert_off[r], rta = c.tri_off[r];
            if (shapes[k].nd != nd || c.tri_off[r + 1] - rta != nt) continue;
            bool same = true;
            for (int64_t t = 0; t < nt && same; ++t)
                for (int d = 0; d < 3 && same; ++d) same = ht[d * T + ta + t] - a == ht[d * T + rta + t] - ra;
            if (same) found = (int)k;
        }
        if (found < 0) {
            double cx = 0, cy = 0, cz = 0;
            for (int64_t j = a; j < a + nd; ++j) {
                cx += hx[j];
                cy += hx[N + j];
                cz += hx[2 * N + j];
            }
            shapes.push_back({m, (int)nd, cx / nd, cy / nd, cz / nd});
            found = (int)shapes.size() - 1;
        }
        shape_of[m] = found;
    }
}

void build(Context &c) {
    cudaStream_t st = c.stream;
    const int64_t N = c.N, M = c.M;
    auto &bp = c.bp;
    std::vector<double> hx(3 * N);
    std::vector<int32_t> ht(3 * (size_t)c.T);
    BEM_CUDA(cudaMemcpyAsync(hx.data(), c.xyz.p, 3 * N * sizeof(double), cudaMemcpyDeviceToHost, st));
    BEM_CUDA(cudaMemcpyAsync(ht.data(), c.tri.p, 3 * (size_t)c.T * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
    BEM_CUDA(cudaStreamSynchronize(st));
    std::vector<BubbleShape> shapes;
    std::vector<int32_t> shape_of;
    find_topologies(c, hx, ht, shapes, shape_of);
    const size_t ns = shapes.size();
    bp.nd.assign(ns, 0);
    bp.inv_off.assign(ns + 1, 0);
    for (size_t k = 0; k < ns; ++k) {
        bp.nd[k] = shapes[k].nd;
        bp.inv_off[k + 1] = bp.inv_off[k] + (int64_t)shapes[k].nd * shapes[k].nd;
    }
    if (bp.inv_off.back() > (int64_t)1 << 30)
        fail(BEM_ERR_ARG, "bubble-block preconditioner: too many distinct bubble meshes (inverse over 8 GiB)");
    // bubbles grouped by shape
    bp.first.assign(ns + 1, 0);
    for (int64_t m = 0; m < M; ++m) bp.first[shape_of[m] + 1] += 1;
    for (size_t k = 0; k < ns; ++k) bp.first[k + 1] += bp.first[k];
    std::vector<int64_t> grouped(M), fill(bp.first.begin(), bp.first.end() - 1);
    for (int64_t m = 0; m < M; ++m) grouped[fill[shape_of[m]]++] = c.vert_off[m];
    bp.bub_voff.resize(M);
    bp.bub_scale.resize(M);
    BEM_CUDA(cudaMemcpyAsync(bp.bub_voff.p, grouped.data(), M * sizeof(int64_t), cudaMemcpyHostToDevice, st));

    bp.inv64.resize(bp.inv_off.back());
    // the tensor-core tables: per shape [3][n_ks][M_pad x 16]
    bp.tc_off.assign(ns + 1, 0);
    for (size_t k = 0; k < ns; ++k) {
        const int64_t nks = div_up(shapes[k].nd, TC_K), Mpad = (int64_t)div_up(shapes[k].nd, BPC_M) * BPC_M;
        bp.tc_off[k + 1] = bp.tc_off[k] + 3 * nks * Mpad * TC_K;
    }
    bp.tcA.resize(bp.tc_off.back());
    int ndmax = 0;
    for (auto &sh : shapes) ndmax = std::max(ndmax, sh.nd);
    DevBuf<double> A, piv;
    DevBuf<int> bad;
    A.resize((size_t)ndmax * ndmax);
    piv.resize(1);
    bad.resize(1);
    BEM_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
    for (size_t k = 0; k < ns; ++k) {
        const BubbleShape &sh = shapes[k];
        const int n = sh.nd;
        const int64_t a = c.vert_off[sh.rep];
        double R = 0.0;  // mean centroid distance of the representative
        for (int i = 0; i < n; ++i) {
            const double dx = hx[a + i] - sh.cx, dy = hx[N + a + i] - sh.cy, dz = hx[2 * N + a + i] - sh.cz;
            R += std::sqrt(dx * dx + dy * dy + dz * dz);
        }
        R /= n;
        k_bp_assemble<<<div_up(n, 128), 128, 0, st>>>(n, N, a, sh.cx, sh.cy, sh.cz, c.xyz.p, c.s.p, c.nrm.p, A.p);
        BEM_LAUNCH_CHECK();
        const dim3 gi((unsigned)div_up(n, 256), (unsigned)n);
        for (int p = 0; p < n; ++p) {
            k_gj_interior<<<gi, 256, 0, st>>>(n, p, A.p, piv.p);
            BEM_LAUNCH_CHECK();
            k_gj_pivot<<<div_up(n, 256), 256, 0, st>>>(n, p, A.p, piv.p, bad.p);
            BEM_LAUNCH_CHECK();
        }
        const size_t cnt = (size_t)n * n;
        k_bp_store<<<(unsigned)std::min<size_t>(div_up((int64_t)cnt, 256), 4096), 256, 0, st>>>(
            cnt, R, A.p, bp.inv64.p + bp.inv_off[k]);
        const int nks = div_up(n, TC_K), Mpad = div_up(n, BPC_M) * BPC_M;
        k_bp_split_inv<<<(unsigned)std::min(div_up((int64_t)Mpad * nks * 2, 256), 4096), 256, 0, st>>>(
            n, nks, Mpad, bp.inv64.p + bp.inv_off[k],
            reinterpret_cast<__nv_bfloat16 *>(bp.tcA.p) + bp.tc_off[k]);
        BEM_LAUNCH_CHECK();
    }
    int hb = 0;
    BEM_CUDA(cudaMemcpyAsync(&hb, bad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    BEM_CUDA(cudaStreamSynchronize(st));
    if (hb) fail(BEM_ERR_MESH, "bubble-block preconditioner: a bubble's single-layer block has a non-positive pivot");
    bp.ready = true;
}

}  // namespace

void block_precond_prepare(Context &c) {
    if (c.M < 1) fail(BEM_ERR_ARG, "the bubble-block preconditioner needs bubbles (vertex offsets)");
    if (!c.bp.ready) build(c);
    auto &bp = c.bp;
    if (c.prm.precision != BEM_PREC_FP64) {
        if (!bp.tc_attr) {
            BEM_CUDA(cudaFuncSetAttribute(k_bp_apply_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)BPC_SMEM));
            bp.tc_attr = true;
        }
        if (c.tc_err.n == 0) {
            c.tc_err.resize(1);
            BEM_CUDA(cudaMemsetAsync(c.tc_err.p, 0, sizeof(int), c.stream));
        }
    }
    for (size_t k = 0; k + 1 < bp.first.size(); ++k) {
        const int64_t nb = bp.first[k + 1] - bp.first[k];
        if (nb == 0) continue;
        k_bp_scales<<<(unsigned)nb, 128, 0, c.stream>>>(bp.nd[k], c.N, bp.bub_voff.p + bp.first[k], c.xyz.p,
                                                        bp.bub_scale.p + bp.first[k]);
        BEM_LAUNCH_CHECK();
    }
}

void block_precond_check(Context &c) {
    if (c.prm.precision == BEM_PREC_FP64 || c.tc_err.n == 0) return;
    int he = 0;
    BEM_CUDA(cudaMemcpyAsync(&he, c.tc_err.p, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
    BEM_CUDA(cudaStreamSynchronize(c.stream));
    if (he) fail(BEM_ERR_TIMEOUT, "tensor-core wait ran out (preconditioner or M2L)");
}

void block_precond_apply(Context &c, const double *y, double *z) {
    auto &bp = c.bp;
    const bool f64 = c.prm.precision == BEM_PREC_FP64;
    for (size_t k = 0; k + 1 < bp.first.size(); ++k) {
        const int64_t nb = bp.first[k + 1] - bp.first[k];
        if (nb == 0) continue;
        const int n = bp.nd[k];
        const int64_t *vo = bp.bub_voff.p + bp.first[k];
        const double *sc = bp.bub_scale.p + bp.first[k];
        if (f64) {
            const dim3 grid((unsigned)div_up(n, BP_TM), (unsigned)div_up(nb, BP_TN));
            k_bp_apply<double><<<grid, BP_THREADS, 0, c.stream>>>(n, bp.inv64.p + bp.inv_off[k], (int)nb, vo, sc, y, z);
        } else {
            const int nks = div_up(n, TC_K), Mpad = div_up(n, BPC_M) * BPC_M;
            const int NBpad = div_up(nb, BPC_N) * BPC_N;
            bp.ys.resize((size_t)3 * nks * NBpad * TC_K);
            __nv_bfloat16 *ys = reinterpret_cast<__nv_bfloat16 *>(bp.ys.p);
            k_bp_split_y<<<(unsigned)std::min(div_up((int64_t)NBpad * nks * 2, 256), 152 * 16), 256, 0, c.stream>>>(
                n, nks, (int)nb, NBpad, vo, y, ys);
            BEM_LAUNCH_CHECK();
            const dim3 grid((unsigned)(Mpad / BPC_M), (unsigned)(NBpad / BPC_N));
            k_bp_apply_tc<<<grid, BPC_THREADS, BPC_SMEM, c.stream>>>(
                n, nks, Mpad, NBpad, (int)nb, reinterpret_cast<const __nv_bfloat16 *>(bp.tcA.p) + bp.tc_off[k], ys, vo,
                sc, z, c.tc_err.p);
        }
        BEM_LAUNCH_CHECK();
    }
}

}  // namespace bem
