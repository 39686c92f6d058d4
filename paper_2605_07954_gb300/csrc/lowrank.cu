// lowrank.cu -- the Jacobi step with the weights factored into separable terms.
//
// A (2r+1) x (2r+1) weight array of rank rho is a sum of rho outer products,
// W[dy][dx] = sum_k c_k[dy] * v_k[dx] (its singular value decomposition).  The
// step of Sec. II-C then splits into rho one-dimensional passes each way:
//     h_k[i][j]   = sum_dx v_k[dx] * u~[i][j+dx]        (along the row)
//     u'[i][j]    = sum_dy sum_k c_k[dy] * h_k[i+dy][j]  (down the column)
// that is 2 * rho * (2r+1) FMAs per point instead of (2r+1)^2: fewer for
// rho < (2r+1)/2 (rank 1..3 of a 7x7 box), more for full-rank weights.  The
// paper cites low-rank tensor-core stencils (LoRAStencil, Sec. II-D) as related
// work; this is the CUDA-core form of the same factorisation.
//
// Host: a one-sided Jacobi SVD of W in FP64, factors c_k = sqrt(s_k) U[:,k],
// v_k = sqrt(s_k) V[:,k] rounded to FP32, numerical rank = the singular
// values above 1e-6 of the largest (or a rank the caller fixes).
//
// Device: one step per launch.  A CTA owns 128 columns and `rows` output rows;
// each thread one column.  Input rows stream through a double-buffered
// shared-memory row of 128 + 2r values (zero or wrapped outside the grid), one
// barrier per row; each thread forms its rho row-pass values and adds them,
// weighted by c_k[dy], into 2r+1 partial sums sliding down its column (the
// arriving row is the last input of output row i - r).
#include <cuda_runtime.h>

#include <cmath>

#include "common.cuh"

namespace gbst {

constexpr int kLrThreads = 128;
constexpr int kLrMaxRank = 2 * kMaxRadius + 1;

struct LowRankParams {
    const float* in;
    float* out;
    long long ny, nx;
    int rows;      // output rows per CTA
    int strips;    // 128-column strips
    int periodic;  // 1: wrap; 0: zero outside the grid
    float col[kLrMaxRank][kLrMaxRank];  // c_k[dy + r]
    float row[kLrMaxRank][kLrMaxRank];  // v_k[dx + r]
};

template <int R, int RHO>
__global__ void __launch_bounds__(kLrThreads) lowrank_step_kernel(const __grid_constant__ LowRankParams p) {
    constexpr int D = 2 * R + 1;
    constexpr int W = kLrThreads + 2 * R;
    __shared__ float buf[2][W];
    const int tid = threadIdx.x;
    const long long ny = p.ny, nx = p.nx;
    const long long x0 = (long long)(blockIdx.x % p.strips) * kLrThreads;
    const long long y0 = (long long)(blockIdx.x / p.strips) * p.rows;
    const long long ylast = y0 + p.rows < ny ? y0 + p.rows : ny;
    const long long j = x0 + tid;

    float acc[D];
#pragma unroll
    for (int m = 0; m < D; ++m) acc[m] = 0.f;
    const long long nsteps = (ylast - y0) + 2 * R;
    const long long nround = (nsteps + D - 1) / D * D;

    auto load = [&](float* dst, long long y) {
        const bool yin = p.periodic || (y >= 0 && y < ny);
        long long yy = y;
        if (p.periodic) yy = ((y % ny) + ny) % ny;
        for (int c = tid; c < W; c += kLrThreads) {
            long long x = x0 - R + c;
            float v = 0.f;
            if (p.periodic) {
                x = ((x % nx) + nx) % nx;
                v = __ldg(p.in + yy * nx + x);
            } else if (yin && x >= 0 && x < nx) {
                v = __ldg(p.in + yy * nx + x);
            }
            dst[c] = v;
        }
    };

    for (long long s0 = 0; s0 < nround; s0 += D) {
#pragma unroll
        for (int jj = 0; jj < D; ++jj) {
            const long long s = s0 + jj;
            const long long y = y0 - R + s;  // the arriving input row
            float* b = buf[s & 1];
            load(b, y);
            __syncthreads();
            float h[RHO];
#pragma unroll
            for (int k = 0; k < RHO; ++k) {
                float t = p.row[k][0] * b[tid];
#pragma unroll
                for (int dx = 1; dx < D; ++dx) t = fmaf(p.row[k][dx], b[tid + dx], t);
                h[k] = t;
            }
            // Row y feeds output row y - dy with weight c_k[dy], dy = -R..R.  The
            // partial sum of output row y_o lives in slot (step of row y_o) mod D;
            // row y arrives at step s, so output y - dy's slot is (s - dy) mod D.
#pragma unroll
            for (int dy = -R; dy <= R; ++dy) {
                const int slot = (jj - dy + 2 * D) % D;
                float t = dy == -R ? 0.f : acc[slot];  // output row y + R starts here
#pragma unroll
                for (int k = 0; k < RHO; ++k) t = fmaf(p.col[k][dy + R], h[k], t);
                acc[slot] = t;
            }
            // output row y - R is complete (its last input row has arrived)
            const long long yo = y - R;
            const int done = (jj - R + 2 * D) % D;
            if (yo >= y0 && yo < ylast && j < nx) p.out[yo * nx + j] = acc[done];
        }
    }
}

// Kernel for rank rho <= 2R+1 (the rank of a (2R+1)-square matrix).
template <int R, int RHO>
static const void* lowrank_pick(int rho) {
    if constexpr (RHO > 2 * R + 1) {
        return nullptr;
    } else {
        if (rho == RHO) return (const void*)lowrank_step_kernel<R, RHO>;
        if constexpr (RHO < 2 * R + 1) return lowrank_pick<R, RHO + 1>(rho);
        return nullptr;
    }
}

template <int R>
static const void* lowrank_kernel_r(int rho) {
    return lowrank_pick<R, 1>(rho);
}

// One-sided Jacobi SVD of the d x d matrix a (row-major, FP64): on return the
// columns of a are U * diag(s) and v holds V, with W = U diag(s) V^T.
static void jacobi_svd(double* a, double* v, int d) {
    for (int i = 0; i < d * d; ++i) v[i] = (i / d == i % d) ? 1.0 : 0.0;
    for (int sweep = 0; sweep < 60; ++sweep) {
        double off = 0.0;
        for (int p = 0; p < d - 1; ++p)
            for (int q = p + 1; q < d; ++q) {
                double al = 0, be = 0, ga = 0;
                for (int i = 0; i < d; ++i) {
                    al += a[i * d + p] * a[i * d + p];
                    be += a[i * d + q] * a[i * d + q];
                    ga += a[i * d + p] * a[i * d + q];
                }
                if (ga == 0.0 || std::fabs(ga) <= 1e-300) continue;
                off = std::fmax(off, std::fabs(ga) / std::sqrt(al * be + 1e-300));
                const double zeta = (be - al) / (2.0 * ga);
                const double t = (zeta >= 0 ? 1.0 : -1.0) / (std::fabs(zeta) + std::sqrt(1.0 + zeta * zeta));
                const double c = 1.0 / std::sqrt(1.0 + t * t), s = c * t;
                for (int i = 0; i < d; ++i) {
                    const double ap = a[i * d + p], aq = a[i * d + q];
                    a[i * d + p] = c * ap - s * aq;
                    a[i * d + q] = s * ap + c * aq;
                    const double vp = v[i * d + p], vq = v[i * d + q];
                    v[i * d + p] = c * vp - s * vq;
                    v[i * d + q] = s * vp + c * vq;
                }
            }
        if (off < 1e-15) break;
    }
}

// Factor W (FP32, (2R+1)^2) into rho separable terms.  rank > 0 fixes rho;
// rank == 0 keeps the singular values above 1e-6 of the largest.  Returns rho
// (0 for an all-zero W) and fills the FP32 factors.
int lowrank_factor(const float* w, int R, int rank, float col[7][7], float row[7][7], double* sv) {
    const int d = 2 * R + 1;
    double a[49], v[49];
    for (int i = 0; i < d * d; ++i) a[i] = w[i];
    jacobi_svd(a, v, d);
    double s[7];
    int order[7];
    for (int k = 0; k < d; ++k) {
        double n = 0;
        for (int i = 0; i < d; ++i) n += a[i * d + k] * a[i * d + k];
        s[k] = std::sqrt(n);
        order[k] = k;
    }
    for (int i = 0; i < d; ++i)  // sort by singular value, descending
        for (int j2 = i + 1; j2 < d; ++j2)
            if (s[order[j2]] > s[order[i]]) {
                const int t = order[i];
                order[i] = order[j2];
                order[j2] = t;
            }
    int rho = 0;
    for (int k = 0; k < d; ++k)
        if (s[order[k]] > 1e-6 * s[order[0]] && s[order[k]] > 0) ++rho;
    if (rank > 0) rho = rank < d ? rank : d;
    for (int k = 0; k < 7; ++k)
        for (int i = 0; i < 7; ++i) col[k][i] = row[k][i] = 0.f;
    for (int k = 0; k < rho; ++k) {
        const int c = order[k];
        const double sk = s[c], rt = std::sqrt(sk);
        for (int i = 0; i < d; ++i) {
            // U[:,c] = a[:,c] / s, so c_k = sqrt(s) U[:,c] = a[:,c] / sqrt(s)
            col[k][i] = sk > 0 ? (float)(a[i * d + c] / rt) : 0.f;
            row[k][i] = (float)(rt * v[i * d + c]);
        }
    }
    if (sv)
        for (int k = 0; k < d; ++k) sv[k] = s[order[k]];
    return rho;
}

const void* get_lowrank_kernel(int R, int rho) {
    switch (R) {
        case 1: return lowrank_kernel_r<1>(rho);
        case 2: return lowrank_kernel_r<2>(rho);
        case 3: return lowrank_kernel_r<3>(rho);
        default: return nullptr;
    }
}

cudaError_t launch_lowrank(const void* fn, const float* src, float* dst, long long ny, long long nx, int periodic,
                           const float col[7][7], const float row[7][7], int sms, cudaStream_t st) {
    LowRankParams lp{};
    lp.in = src;
    lp.out = dst;
    lp.ny = ny;
    lp.nx = nx;
    lp.periodic = periodic;
    lp.strips = (int)((nx + kLrThreads - 1) / kLrThreads);
    // about 8 CTAs per SM; at least 16 output rows per CTA
    long long tiles = (long long)sms * 8 / lp.strips;
    if (tiles < 1) tiles = 1;
    long long rows = (ny + tiles - 1) / tiles;
    if (rows < 16) rows = 16;
    lp.rows = (int)rows;
    const long long ty = (ny + rows - 1) / rows;
    for (int k = 0; k < 7; ++k)
        for (int i = 0; i < 7; ++i) {
            lp.col[k][i] = col[k][i];
            lp.row[k][i] = row[k][i];
        }
    void* args[] = {&lp};
    return cudaLaunchKernel(fn, dim3((unsigned)(lp.strips * ty)), dim3(kLrThreads), args, 0, st);
}

}  // namespace gbst
