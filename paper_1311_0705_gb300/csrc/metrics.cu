// Grid-quality metrics of Sect. 3.2 on the device: the true density rho_t
// of the analytic model at points, the true optical depth tau_t along paths
// by adaptive Gauss-Kronrod quadrature, and the two-pass FP64 statistics
// (mean, population standard deviation) of rho_t - rho_g and tau_t - tau_g.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "hg_internal.h"

namespace hg {
hg_status cuda_err(cudaError_t e, const char *what);
int sm_count();

struct DevModel {
    int32_t kind;
    int32_t n_table;
    double p[8];
    const double *table;
    double lo[3], hi[3];
};

__device__ double rho_true(const DevModel &m, double x, double y, double z) {
    switch (m.kind) {
    case HG_MODEL_CONST:
        return m.p[0];
    case HG_MODEL_DISK: {
        const double R = sqrt(x * x + y * y);
        return m.p[0] * exp(-(R / m.p[1]) - (fabs(z) / m.p[2]));
    }
    case HG_MODEL_TORUS: {
        const double s = sqrt(x * x + y * y) - m.p[0];
        double v = (s * s + z * z < m.p[1] * m.p[1]) ? m.p[2] : 0.0;
        const float xf = (float)x, yf = (float)y, zf = (float)z;
        for (int j = 0; j < m.n_table; j++) {
            const double *c = m.table + 5 * j;
            // single-precision pre-filter with a wide margin, exact test in FP64
            const float dxf = xf - (float)c[0], dyf = yf - (float)c[1], dzf = zf - (float)c[2];
            const float sf = (float)c[3];
            if (dxf * dxf + dyf * dyf + dzf * dzf > 25.5f * sf * sf + 1e-30f) continue;
            const double dx = x - c[0], dy = y - c[1], dz = z - c[2];
            const double r2 = dx * dx + dy * dy + dz * dz;
            const double s2 = c[3] * c[3];
            if (r2 < 25.0 * s2) v += c[4] * exp(-0.5 * (r2 / s2));
        }
        return v;
    }
    case HG_MODEL_DYADIC: {
        const int L = (int)m.p[0];
        const long long n = 1LL << L;
        const double pos[3] = {x, y, z};
        long long ix[3];
        for (int a = 0; a < 3; a++) {
            long long q = (long long)floor((pos[a] - m.lo[a]) / (m.hi[a] - m.lo[a]) * (double)n);
            ix[a] = q < 0 ? 0 : (q > n - 1 ? n - 1 : q);
        }
        return m.table[ix[0] + n * (ix[1] + n * ix[2])];
    }
    }
    return 0.0;
}

__global__ void model_density_kernel(const DevModel m, int64_t n, const double *__restrict__ pts, double *rho) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        rho[i] = rho_true(m, pts[3 * i], pts[3 * i + 1], pts[3 * i + 2]);
}

// 15-point Kronrod abscissae/weights and the embedded 7-point Gauss weights on [-1, 1].
__constant__ double c_xgk[8] = {0.991455371120812639206854697526329, 0.949107912342758524526189684047851,
                                0.864864423359769072789712788640926, 0.741531185599394439863864773280788,
                                0.586087235467691130294144845693013, 0.405845151377397166906606412076961,
                                0.207784955007898467600689403773245, 0.0};
__constant__ double c_wgk[8] = {0.022935322010529224963732008058970, 0.063092092629978553290700663189204,
                                0.104790010322250183839876322541518, 0.140653259715525918745189590510238,
                                0.169004726639267902826583426598550, 0.190350578064785409913256402421014,
                                0.204432940075298892414161999234649, 0.209482141084727828012999174891714};
__constant__ double c_wg[4] = {0.129484966168869693270611432679082, 0.279705391489276667901467771423780,
                               0.381830050505118944950369775488975, 0.417959183673469387755102040816327};

__device__ __forceinline__ double ray_rho(const DevModel &m, const double *o, const double *k, double t) {
    return rho_true(m, o[0] + k[0] * t, o[1] + k[1] * t, o[2] + k[2] * t);
}

__device__ void gk15(const DevModel &m, const double *o, const double *k, double a, double b, double *res,
                     double *err) {
    const double c = 0.5 * (a + b), h = 0.5 * (b - a);
    const double fc = ray_rho(m, o, k, c);
    double rk = fc * c_wgk[7], rg = fc * c_wg[3];
#pragma unroll
    for (int j = 0; j < 7; j++) {
        const double x = h * c_xgk[j];
        const double f1 = ray_rho(m, o, k, c - x), f2 = ray_rho(m, o, k, c + x);
        rk += c_wgk[j] * (f1 + f2);
        if (j & 1) rg += c_wg[j / 2] * (f1 + f2);
    }
    *res = rk * h;
    *err = fabs((rk - rg) * h);
}

// Adaptive bisection with an explicit stack, left half first (the order of
// a recursive depth-first integrator).
__device__ double adapt(const DevModel &m, const double *o, const double *k, double a, double b, double rtol) {
    constexpr int kStack = 64;
    double sa[kStack], sb[kStack];
    int sd[kStack];
    int top = 0;
    sa[0] = a;
    sb[0] = b;
    sd[0] = 0;
    top = 1;
    double total = 0.0;
    while (top > 0) {
        top--;
        const double x0 = sa[top], x1 = sb[top];
        const int dep = sd[top];
        double r, e;
        gk15(m, o, k, x0, x1, &r, &e);
        if (dep >= 60 || e <= rtol * fabs(r) || e < 1e-300 || !(x1 > x0) || top + 2 > kStack) {
            total += r;
            continue;
        }
        const double xm = 0.5 * (x0 + x1);
        sa[top] = xm;
        sb[top] = x1;
        sd[top] = dep + 1;
        sa[top + 1] = x0;
        sb[top + 1] = xm;
        sd[top + 1] = dep + 1;
        top += 2;
    }
    return total;
}

__device__ __forceinline__ double horner(const double *c, int deg, double t) {
    double v = c[deg];
    for (int j = deg - 1; j >= 0; j--) v = v * t + c[j];
    return v;
}

// Real roots in (a, b) of a polynomial of degree <= 4, from the roots of its
// successive derivatives (each splits the interval into monotone pieces
// that are bisected).
__device__ int poly_roots4(const double *c4, double a, double b, double *roots) {
    double der[5][5];
    for (int j = 0; j <= 4; j++) der[0][j] = c4[j];
    for (int d = 1; d <= 4; d++)
        for (int j = 0; j <= 4 - d; j++) der[d][j] = (j + 1) * der[d - 1][j + 1];
    double crit[6];
    int nc = 0;
    for (int d = 3; d >= 0; d--) {
        const double *c = der[d];
        int deg = 4 - d;
        while (deg > 0 && c[deg] == 0.0) deg--;
        double edges[6];
        int ne = 0;
        edges[ne++] = a;
        for (int j = 0; j < nc; j++) edges[ne++] = crit[j];
        edges[ne++] = b;
        double out[5];
        int nr = 0;
        if (deg >= 1) {
            for (int j = 0; j + 1 < ne; j++) {
                double lo = edges[j], hi = edges[j + 1];
                double flo = horner(c, deg, lo);
                const double fhi = horner(c, deg, hi);
                if (flo == 0.0) {
                    if (lo > a) out[nr++] = lo;
                    continue;
                }
                if ((flo < 0.0) == (fhi < 0.0)) continue;
                for (int it = 0; it < 200; it++) {
                    const double mid = 0.5 * (lo + hi);
                    if (mid <= lo || mid >= hi) break;
                    const double fm = horner(c, deg, mid);
                    if ((fm < 0.0) == (flo < 0.0)) {
                        lo = mid;
                        flo = fm;
                    } else {
                        hi = mid;
                    }
                }
                out[nr++] = 0.5 * (lo + hi);
            }
        }
        nc = nr;
        for (int j = 0; j < nr; j++) crit[j] = out[j];
    }
    for (int j = 0; j < nc; j++) roots[j] = crit[j];
    return nc;
}

constexpr int kMaxBreak = 160;

__device__ __forceinline__ void add_bp(double *bp, int &nb, double t, double L) {
    if (t > 0.0 && t < L && nb < kMaxBreak - 1) bp[nb++] = t;
}

__global__ void model_tau_kernel(const DevModel m, int64_t n, const double *__restrict__ O,
                                 const double *__restrict__ K, const double *__restrict__ len, double kappa,
                                 double rtol, double *tau) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double o[3] = {O[3 * i], O[3 * i + 1], O[3 * i + 2]};
        const double k[3] = {K[3 * i], K[3 * i + 1], K[3 * i + 2]};
        const double L = len[i];
        double bp[kMaxBreak];
        int nb = 0;
        bp[nb++] = 0.0;
        if (m.kind == HG_MODEL_DISK) {
            if (k[2] != 0.0) add_bp(bp, nb, -o[2] / k[2], L);
            const double kk = k[0] * k[0] + k[1] * k[1];
            if (kk > 0.0) add_bp(bp, nb, -(o[0] * k[0] + o[1] * k[1]) / kk, L);
        } else if (m.kind == HG_MODEL_TORUS) {
            const double R = m.p[0], r = m.p[1];
            const double A = k[0] * k[0] + k[1] * k[1] + k[2] * k[2];
            const double B = 2.0 * (o[0] * k[0] + o[1] * k[1] + o[2] * k[2]);
            const double C = o[0] * o[0] + o[1] * o[1] + o[2] * o[2] + R * R - r * r;
            const double D = k[0] * k[0] + k[1] * k[1];
            const double E = 2.0 * (o[0] * k[0] + o[1] * k[1]);
            const double F = o[0] * o[0] + o[1] * o[1];
            const double c4[5] = {C * C - 4.0 * R * R * F, 2.0 * B * C - 4.0 * R * R * E,
                                  B * B + 2.0 * A * C - 4.0 * R * R * D, 2.0 * A * B, A * A};
            double roots[5];
            const int nr = poly_roots4(c4, 0.0, L, roots);
            for (int j = 0; j < nr; j++) add_bp(bp, nb, roots[j], L);
            for (int j = 0; j < m.n_table; j++) {
                const double *cl = m.table + 5 * j;
                const double w0 = o[0] - cl[0], w1 = o[1] - cl[1], w2 = o[2] - cl[2];
                const double b2 = w0 * k[0] + w1 * k[1] + w2 * k[2];
                const double cc = w0 * w0 + w1 * w1 + w2 * w2 - 25.0 * cl[3] * cl[3];
                const double disc = b2 * b2 - A * cc;
                if (disc <= 0.0) continue;
                const double sq = sqrt(disc);
                add_bp(bp, nb, (-b2 - sq) / A, L);
                add_bp(bp, nb, (-b2 + sq) / A, L);
                add_bp(bp, nb, -b2 / A, L);
            }
        } else if (m.kind == HG_MODEL_DYADIC) {
            const long long nn = 1LL << (int)m.p[0];
            for (int a = 0; a < 3; a++) {
                if (k[a] == 0.0) continue;
                for (long long j = 1; j < nn; j++) {
                    const double pl = m.lo[a] + (m.hi[a] - m.lo[a]) * ((double)j / (double)nn);
                    add_bp(bp, nb, (pl - o[a]) / k[a], L);
                }
            }
        }
        bp[nb++] = L;
        // insertion sort (short lists)
        for (int a = 1; a < nb; a++) {
            const double v = bp[a];
            int b = a - 1;
            while (b >= 0 && bp[b] > v) {
                bp[b + 1] = bp[b];
                b--;
            }
            bp[b + 1] = v;
        }
        double tot = 0.0;
        for (int j = 0; j + 1 < nb; j++)
            if (bp[j + 1] > bp[j]) tot += adapt(m, o, k, bp[j], bp[j + 1], rtol);
        tau[i] = kappa * tot;
    }
}

// Deterministic two-pass statistics: per-block partials, then one block.
__device__ __forceinline__ double block_sum(double v, double *sh) {
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double s = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) s += sh[w];
    __syncthreads();
    return s;
}

__global__ void diff_partial(int64_t n, const double *__restrict__ a, const double *__restrict__ b,
                             const double *mean_src, double *part) {
    __shared__ double sh[32];
    const double mu = mean_src ? mean_src[1] : 0.0;
    double s = 0.0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double x = a[i] - b[i];
        if (mean_src) {
            const double y = x - mu;
            s += y * y;
        } else {
            s += x;
        }
    }
    s = block_sum(s, sh);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void diff_final(int64_t n, int nparts, const double *part, double *out, int stage) {
    __shared__ double sh[32];
    double s = 0.0;
    for (int i = threadIdx.x; i < nparts; i += blockDim.x) s += part[i];
    s = block_sum(s, sh);
    if (threadIdx.x == 0) {
        if (stage == 0) {
            out[0] = (double)n;
            out[1] = n ? s / (double)n : 0.0;
        } else {
            out[2] = n ? sqrt(s / (double)n) : 0.0;
        }
    }
}

}  // namespace hg

struct hg_dmodel {
    hg::DevModel m;
    void *d_table = nullptr;
};

using namespace hg;

extern "C" hg_status hg_load_model(const hg_model *model, hg_dmodel **out) {
    if (!model || !out) { set_error("hg_load_model: null argument"); return HG_EINVAL; }
    *out = nullptr;
    if (model->kind < HG_MODEL_CONST || model->kind > HG_MODEL_DYADIC || model->n_table < 0 ||
        (model->n_table > 0 && !model->table)) {
        set_error("hg_load_model: bad model");
        return HG_EINVAL;
    }
    hg_dmodel *dm = new hg_dmodel();
    dm->m.kind = model->kind;
    dm->m.n_table = model->n_table;
    for (int j = 0; j < 8; j++) dm->m.p[j] = model->p[j];
    for (int a = 0; a < 3; a++) {
        dm->m.lo[a] = model->lo[a];
        dm->m.hi[a] = model->hi[a];
    }
    const size_t per = (model->kind == HG_MODEL_TORUS) ? 5 : 1;
    const size_t bytes = std::max<size_t>(8, (size_t)model->n_table * per * sizeof(double));
    cudaError_t e = cudaMalloc(&dm->d_table, bytes);
    if (e == cudaSuccess && model->n_table > 0)
        e = cudaMemcpy(dm->d_table, model->table, (size_t)model->n_table * per * sizeof(double),
                       cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
        hg_free_model(dm);
        return cuda_err(e, "hg_load_model");
    }
    dm->m.table = static_cast<const double *>(dm->d_table);
    *out = dm;
    return HG_OK;
}

extern "C" void hg_free_model(hg_dmodel *m) {
    if (!m) return;
    if (m->d_table) cudaFree(m->d_table);
    delete m;
}

extern "C" hg_status hg_model_density(const hg_dmodel *m, int64_t n, const double *pts, double *rho,
                                      hg_stream stream) {
    if (!m || n < 0 || (n > 0 && (!pts || !rho))) { set_error("hg_model_density: bad arguments"); return HG_EINVAL; }
    if (n == 0) return HG_OK;
    const int64_t blocks = std::min<int64_t>((n + 255) / 256, (int64_t)sm_count() * 8);
    model_density_kernel<<<(unsigned)blocks, 256, 0, (cudaStream_t)stream>>>(m->m, n, pts, rho);
    note_launches(1);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HG_OK : cuda_err(e, "model density launch");
}

extern "C" hg_status hg_model_tau(const hg_dmodel *m, int64_t n, const double *o, const double *d,
                                  const double *len, double kappa, double rtol, double *tau, hg_stream stream) {
    if (!m || n < 0 || (n > 0 && (!o || !d || !len || !tau)) || !(rtol > 0.0)) {
        set_error("hg_model_tau: bad arguments");
        return HG_EINVAL;
    }
    if (n == 0) return HG_OK;
    const int block = 128;
    const int64_t blocks = std::min<int64_t>((n + block - 1) / block, (int64_t)sm_count() * 16);
    model_tau_kernel<<<(unsigned)blocks, block, 0, (cudaStream_t)stream>>>(m->m, n, o, d, len, kappa, rtol, tau);
    note_launches(1);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HG_OK : cuda_err(e, "model tau launch");
}

extern "C" hg_status hg_diff_stats(int64_t n, const double *a, const double *b, double *out, hg_stream stream) {
    if (n < 0 || !out || (n > 0 && (!a || !b))) { set_error("hg_diff_stats: bad arguments"); return HG_EINVAL; }
    cudaStream_t s = (cudaStream_t)stream;
    const int block = 256;
    const int parts = (int)std::max<int64_t>(1, std::min<int64_t>((n + block - 1) / block, (int64_t)sm_count() * 4));
    double *part = nullptr;
    cudaError_t e = cudaMallocAsync((void **)&part, (size_t)parts * sizeof(double), s);
    if (e != cudaSuccess) return cuda_err(e, "diff stats scratch");
    diff_partial<<<parts, block, 0, s>>>(n, a, b, nullptr, part);
    diff_final<<<1, 1024, 0, s>>>(n, parts, part, out, 0);
    diff_partial<<<parts, block, 0, s>>>(n, a, b, out, part);
    diff_final<<<1, 1024, 0, s>>>(n, parts, part, out, 1);
    note_launches(4);
    e = cudaGetLastError();
    cudaFreeAsync(part, s);
    return e == cudaSuccess ? HG_OK : cuda_err(e, "diff stats launch");
}
