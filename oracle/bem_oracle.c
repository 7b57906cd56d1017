/*
 * Plain FP64 CPU reference for the collocation boundary-element operators of the
 * bubble-dynamics method (Gumerov, Pityuk, Abramova, Akhatov, arXiv:1905.01341).
 *
 * TEST INFRASTRUCTURE ONLY. This file is part of the oracle: only the test-suite, the
 * smoke check and the CPU-baseline leg of the benchmark may load it. The product (the
 * CUDA library) shares no code, header, table or helper with it.
 *
 * What it computes, in the paper's notation:
 *  - vertex weights and normals, Section 3.2 "Non-singular integrals", Eq. (ns1):
 *      s_j = (1/3) sum_{S_k containing r_j} A_k,
 *      m_j = sum_{S_k containing r_j} N_k A_k,  n_j = m_j / |m_j|;
 *  - the off-diagonal single- and double-layer sums of Eq. (ns1) with the kernels of
 *    Eq. (2.13):
 *      (L_off X)_i = sum_{j != i} s_j X_j / (4 pi |r_i - r_j|),
 *      (M_off X)_i = sum_{j != i} s_j X_j n_j.(r_i - r_j) / (4 pi |r_i - r_j|^3),
 *    combined as in Eq. (3.27): out_i = f (L_off xL)_i + g (M_off xM)_i.
 * Every sum over j is a plain loop in index order with Neumaier compensation, so the
 * result is the exact discrete sum up to FP64 rounding. No blocking, no reordering.
 */
#include <math.h>
#include <stdint.h>
#include <stddef.h>

#define ORACLE_PI 3.14159265358979323846

/* Neumaier-compensated accumulator. */
typedef struct {
    double s, c;
} acc_t;

static inline void acc_add(acc_t *a, double v)
{
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v))
        a->c += (a->s - t) + v;
    else
        a->c += (v - t) + a->s;
    a->s = t;
}

static inline double acc_get(const acc_t *a) { return a->s + a->c; }

/*
 * Eq. (ns1): per-vertex weight s_j and unit normal n_j from the triangles touching it.
 * xyz: [N][3]; tri: [T][3] (counter-clockwise seen from the liquid, so the right-hand
 * normal N_k points out of the bubble, Section 3.4); outputs s: [N], nrm: [N][3].
 * Returns 0, or -1 if a vertex index is out of range, or -2 if some vertex touches no
 * triangle or has a zero area-weighted normal.
 */
int oracle_vertex_geometry(int64_t N, const double *xyz, int64_t T, const int32_t *tri,
                           double *s, double *nrm)
{
    for (int64_t j = 0; j < N; ++j) {
        s[j] = 0.0;
        nrm[3 * j] = nrm[3 * j + 1] = nrm[3 * j + 2] = 0.0;
    }
    for (int64_t k = 0; k < T; ++k) {
        int32_t a = tri[3 * k], b = tri[3 * k + 1], c = tri[3 * k + 2];
        if (a < 0 || b < 0 || c < 0 || a >= N || b >= N || c >= N)
            return -1;
        double e1[3], e2[3], cr[3];
        for (int d = 0; d < 3; ++d) {
            e1[d] = xyz[3 * b + d] - xyz[3 * a + d];
            e2[d] = xyz[3 * c + d] - xyz[3 * a + d];
        }
        cr[0] = e1[1] * e2[2] - e1[2] * e2[1];
        cr[1] = e1[2] * e2[0] - e1[0] * e2[2];
        cr[2] = e1[0] * e2[1] - e1[1] * e2[0];
        /* N_k A_k = half the cross product; A_k its length. */
        double NA[3] = {0.5 * cr[0], 0.5 * cr[1], 0.5 * cr[2]};
        double A = sqrt(NA[0] * NA[0] + NA[1] * NA[1] + NA[2] * NA[2]);
        int32_t v[3] = {a, b, c};
        for (int q = 0; q < 3; ++q) {
            s[v[q]] += A / 3.0;
            for (int d = 0; d < 3; ++d)
                nrm[3 * v[q] + d] += NA[d];
        }
    }
    for (int64_t j = 0; j < N; ++j) {
        double mx = nrm[3 * j], my = nrm[3 * j + 1], mz = nrm[3 * j + 2];
        double len = sqrt(mx * mx + my * my + mz * mz);
        if (!(s[j] > 0.0) || !(len > 0.0))
            return -2;
        nrm[3 * j] = mx / len;
        nrm[3 * j + 1] = my / len;
        nrm[3 * j + 2] = mz / len;
    }
    return 0;
}

/*
 * Eq. (ns1)/(3.27): out[r] = f (L_off xL)_i + g (M_off xM)_i for receivers i = recv[r]
 * (or i = r when recv is NULL, nrecv = N). Sources are all N vertices except i itself.
 * xL or xM may be NULL when the matching coefficient f or g is zero.
 * OpenMP splits receivers across threads; each receiver's sum runs over j in order.
 */
void oracle_offdiag_apply(int64_t N, const double *xyz, const double *s, const double *nrm,
                          double f, const double *xL, double g, const double *xM,
                          int64_t nrecv, const int64_t *recv, double *out)
{
    const double inv4pi = 1.0 / (4.0 * ORACLE_PI);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t r = 0; r < nrecv; ++r) {
        int64_t i = recv ? recv[r] : r;
        double xi = xyz[3 * i], yi = xyz[3 * i + 1], zi = xyz[3 * i + 2];
        acc_t acc = {0.0, 0.0};
        for (int64_t j = 0; j < N; ++j) {
            if (j == i)
                continue;
            double dx = xi - xyz[3 * j], dy = yi - xyz[3 * j + 1], dz = zi - xyz[3 * j + 2];
            double r2 = dx * dx + dy * dy + dz * dz;
            double rr = sqrt(r2);
            double term = 0.0;
            if (f != 0.0)
                term += f * xL[j] / rr;                                   /* G, Eq. (2.13) */
            if (g != 0.0)
                term += g * xM[j] * (nrm[3 * j] * dx + nrm[3 * j + 1] * dy + nrm[3 * j + 2] * dz)
                        / (rr * r2);                                        /* dG/dn', Eq. (2.13) */
            acc_add(&acc, s[j] * term * inv4pi);
        }
        out[r] = acc_get(&acc);
    }
}

/*
 * Dense assembly of the off-diagonal matrices of Eq. (ns1) for small N:
 * Lm[i*N+j] = s_j G(r_i, r_j), Mm[i*N+j] = s_j dG/dn_j(r_i, r_j), zero diagonal.
 */
void oracle_offdiag_dense(int64_t N, const double *xyz, const double *s, const double *nrm,
                          double *Lm, double *Mm)
{
    const double inv4pi = 1.0 / (4.0 * ORACLE_PI);
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < N; ++i) {
        for (int64_t j = 0; j < N; ++j) {
            if (j == i) {
                Lm[i * N + j] = 0.0;
                Mm[i * N + j] = 0.0;
                continue;
            }
            double dx = xyz[3 * i] - xyz[3 * j], dy = xyz[3 * i + 1] - xyz[3 * j + 1],
                   dz = xyz[3 * i + 2] - xyz[3 * j + 2];
            double r2 = dx * dx + dy * dy + dz * dz;
            double rr = sqrt(r2);
            Lm[i * N + j] = s[j] * inv4pi / rr;
            Mm[i * N + j] = s[j] * inv4pi *
                            (nrm[3 * j] * dx + nrm[3 * j + 1] * dy + nrm[3 * j + 2] * dz) / (rr * r2);
        }
    }
}

/* Number of OpenMP threads the sums use (1 when built without OpenMP). */
int oracle_num_threads(void)
{
#ifdef _OPENMP
    extern int omp_get_max_threads(void);
    return omp_get_max_threads();
#else
    return 1;
#endif
}
