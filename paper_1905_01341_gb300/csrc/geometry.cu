// Vertex weights and normals of the one-point vertex quadrature, Section 3.2, Eq. (ns1):
//   s_j = (1/3) sum_{S_k containing r_j} A_k,   m_j = sum_{S_k containing r_j} N_k A_k,
//   n_j = m_j / |m_j|.
// A vertex -> triangle CSR (triangle ids sorted per vertex) makes every sum run in a fixed
// order, so results do not depend on scheduling.
#include "internal.h"

namespace bem {
namespace {

__global__ void k_count_corners(int64_t T, const int32_t *__restrict__ tri, int64_t N,
                                int32_t *__restrict__ cnt, int *__restrict__ bad) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= T) return;
    for (int c = 0; c < 3; ++c) {
        int32_t v = tri[c * T + k];
        if (v < 0 || v >= N) {
            atomicOr(bad, 1);
            continue;
        }
        atomicAdd(&cnt[v], 1);
    }
}

__global__ void k_fill_corners(int64_t T, const int32_t *__restrict__ tri, int64_t N,
                               const int32_t *__restrict__ off, int32_t *__restrict__ cursor,
                               int32_t *__restrict__ v2t) {
    int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= T) return;
    for (int c = 0; c < 3; ++c) {
        int32_t v = tri[c * T + k];
        if (v < 0 || v >= N) continue;
        int slot = atomicAdd(&cursor[v], 1);
        v2t[off[v] + slot] = (int32_t)k;
    }
}

// Sort every vertex's triangle list (short: the valence) so sums run in triangle order.
__global__ void k_sort_lists(int64_t N, const int32_t *__restrict__ off, int32_t *__restrict__ v2t) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= N) return;
    int a = off[j], b = off[j + 1];
    for (int i = a + 1; i < b; ++i) {
        int32_t x = v2t[i];
        int k = i - 1;
        while (k >= a && v2t[k] > x) {
            v2t[k + 1] = v2t[k];
            --k;
        }
        v2t[k + 1] = x;
    }
}

// Eq. (ns1), per triangle: N_k A_k (half the cross product of the edges) and A_k / 3, stored
// as the pairs (x, y), (z, A_k / 3); computed once per triangle instead of once per corner.
__global__ void k_tri_area_vectors(int64_t T, int64_t N, const double *__restrict__ xyz,
                                   const int32_t *__restrict__ tri, double2 *__restrict__ av) {
    const int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (k >= T) return;
    const double *X = xyz, *Y = xyz + N, *Z = xyz + 2 * N;
    const int32_t a = tri[k], b = tri[T + k], c = tri[2 * T + k];
    const double e1x = X[b] - X[a], e1y = Y[b] - Y[a], e1z = Z[b] - Z[a];
    const double e2x = X[c] - X[a], e2y = Y[c] - Y[a], e2z = Z[c] - Z[a];
    const double nax = 0.5 * (e1y * e2z - e1z * e2y);
    const double nay = 0.5 * (e1z * e2x - e1x * e2z);
    const double naz = 0.5 * (e1x * e2y - e1y * e2x);
    const double A = sqrt(nax * nax + nay * nay + naz * naz);
    av[2 * k] = make_double2(nax, nay);
    av[2 * k + 1] = make_double2(naz, A / 3.0);
}

// Eq. (ns1) per vertex: s_j = sum of A_k / 3 and n_j = m_j / |m_j|, m_j = sum of N_k A_k over the
// vertex's triangles in vertex-to-triangle list order.
__global__ void k_vertex_geometry(int64_t N, const double2 *__restrict__ av, const int32_t *__restrict__ off,
                                  const int32_t *__restrict__ v2t, double *__restrict__ s,
                                  double *__restrict__ nrm, int *__restrict__ bad) {
    int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (j >= N) return;
    double sj = 0.0, mx = 0.0, my = 0.0, mz = 0.0;
    for (int t = off[j]; t < off[j + 1]; ++t) {
        const int64_t k = v2t[t];
        const double2 u = av[2 * k], w = av[2 * k + 1];
        sj += w.y;
        mx += u.x;
        my += u.y;
        mz += w.x;
    }
    double len = sqrt(mx * mx + my * my + mz * mz);
    if (!(sj > 0.0) || !(len > 0.0)) {
        atomicOr(bad, 2);
        len = 1.0;
    }
    s[j] = sj;
    nrm[j] = mx / len;
    nrm[N + j] = my / len;
    nrm[2 * N + j] = mz / len;
}

}  // namespace

void build_vertex_triangle_csr(Context &c) {
    cudaStream_t st = c.stream;
    DevBuf<int32_t> cnt, cursor;
    DevBuf<int> bad;
    cnt.resize(c.N + 1);
    cursor.resize(c.N);
    bad.resize(1);
    BEM_CUDA(cudaMemsetAsync(cnt.p, 0, (c.N + 1) * sizeof(int32_t), st));
    BEM_CUDA(cudaMemsetAsync(cursor.p, 0, c.N * sizeof(int32_t), st));
    BEM_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
    int tb = 256;
    k_count_corners<<<div_up(c.T, tb), tb, 0, st>>>(c.T, c.tri.p, c.N, cnt.p, bad.p);
    BEM_LAUNCH_CHECK();
    c.v2t_off.resize(c.N + 1);
    exclusive_scan_i32(cnt.p, c.v2t_off.p, c.N + 1, nullptr, st);
    c.v2t.resize(3 * c.T);
    k_fill_corners<<<div_up(c.T, tb), tb, 0, st>>>(c.T, c.tri.p, c.N, c.v2t_off.p, cursor.p, c.v2t.p);
    BEM_LAUNCH_CHECK();
    k_sort_lists<<<div_up(c.N, tb), tb, 0, st>>>(c.N, c.v2t_off.p, c.v2t.p);
    BEM_LAUNCH_CHECK();
    int hbad = 0;
    BEM_CUDA(cudaMemcpyAsync(&hbad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    BEM_CUDA(cudaStreamSynchronize(st));
    if (hbad) fail(BEM_ERR_MESH, "triangle vertex index out of range");
}

void compute_vertex_geometry(Context &c) {
    cudaStream_t st = c.stream;
    DevBuf<int> &bad = c.chk[2];
    bad.resize(1);
    BEM_CUDA(cudaMemsetAsync(bad.p, 0, sizeof(int), st));
    c.s.resize(c.N);
    c.nrm.resize(3 * c.N);
    int tb = 256;
    c.tri_tmp.resize(2 * (size_t)c.T);
    if (c.T > 0) {
        k_tri_area_vectors<<<div_up(c.T, tb), tb, 0, st>>>(c.T, c.N, c.xyz.p, c.tri.p, c.tri_tmp.p);
        BEM_LAUNCH_CHECK();
    }
    k_vertex_geometry<<<div_up(c.N, tb), tb, 0, st>>>(c.N, c.tri_tmp.p, c.v2t_off.p, c.v2t.p, c.s.p, c.nrm.p,
                                                      bad.p);
    BEM_LAUNCH_CHECK();
    int hbad = 0;
    BEM_CUDA(cudaMemcpyAsync(&hbad, bad.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    BEM_CUDA(cudaStreamSynchronize(st));
    if (hbad) fail(BEM_ERR_MESH, "vertex without triangles or with zero area-weighted normal");
}

}  // namespace bem
