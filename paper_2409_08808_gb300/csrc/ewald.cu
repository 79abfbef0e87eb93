// Ewald pair matrix J of a periodic supercell (Section "Cluster Expansion of
// Coulomb Energy": the pairwise expansion is exact for point charges, and its
// coefficients are Ewald energies).  FP64 throughout.
//
//   J_ij = ke/2 [ sum'_n erfc(alpha|d+n|)/|d+n|                    (real space)
//               + (4 pi / V) sum_{0<|k|<=kcut} e^{-k^2/4a^2}/k^2 cos(k.d)  (reciprocal)
//               - (2 alpha / sqrt(pi)) delta_ij - pi / (V alpha^2) ]  (self, background)
//
// GPU layout of the work:
//   1. k_geometry: reciprocal basis B = 2 pi A^-T and V (one thread).
//   2. k_kvectors: the half space of reciprocal vectors inside the cutoff,
//      compacted in index order by one block, with weights
//      w = ke (4 pi / V) e^{-k^2/4a^2} / k^2 (the half space counts k and -k).
//   3. k_struct_factor: X = [sqrt(w) cos(k.r_i) | sqrt(w) sin(k.r_i)]  (N x 2K).
//   4. k_syrk_f64: J_rec = X X^T on the lower block triangle (a dense FP64
//      contraction; cos a cos b + sin a sin b = cos(a - b)).
//   5. k_real_space: per pair i <= j the image sum, self and background terms,
//      plus J_rec; writes J_ij and J_ji (exactly symmetric result).
#include <math.h>

#include "common.cuh"

namespace {

constexpr double kPi = 3.14159265358979323846;

// Four doubles, 32-byte aligned (k-vector with its weight, or image translation with a flag).
struct __align__(32) Vec4d {
    double x, y, z, w;
};

struct Geom {
    double A[9];
    double B[9];
    double V;
};

__global__ void k_geometry(const double* __restrict__ A_in, Geom* __restrict__ g)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double A[9];
    for (int t = 0; t < 9; ++t) A[t] = A_in[t];
    // cross products of lattice rows
    double c23[3] = {A[4] * A[8] - A[5] * A[7], A[5] * A[6] - A[3] * A[8], A[3] * A[7] - A[4] * A[6]};
    double c31[3] = {A[7] * A[2] - A[8] * A[1], A[8] * A[0] - A[6] * A[2], A[6] * A[1] - A[7] * A[0]};
    double c12[3] = {A[1] * A[5] - A[2] * A[4], A[2] * A[3] - A[0] * A[5], A[0] * A[4] - A[1] * A[3]};
    double vol = A[0] * c23[0] + A[1] * c23[1] + A[2] * c23[2];
    for (int d = 0; d < 3; ++d) {
        g->B[0 + d] = 2.0 * kPi * c23[d] / vol;
        g->B[3 + d] = 2.0 * kPi * c31[d] / vol;
        g->B[6 + d] = 2.0 * kPi * c12[d] / vol;
    }
    for (int t = 0; t < 9; ++t) g->A[t] = A[t];
    g->V = fabs(vol);
}

// One block: visit the index box m1 in [0, M1], m2 in [-M2, M2], m3 in [-M3, M3]
// in linear order, keep the half space (m1 > 0, or m1 == 0 and m2 > 0, or
// m1 == m2 == 0 and m3 > 0) with |k| <= kcut, compact with a block scan.
__global__ void __launch_bounds__(1024) k_kvectors(const Geom* __restrict__ g, int M1, int M2, int M3, double kcut,
                                                   double alpha, double ke, Vec4d* __restrict__ kv,
                                                   int* __restrict__ count)
{
    __shared__ int warp_sums[32];
    __shared__ int base;
    if (threadIdx.x == 0) base = 0;
    __syncthreads();
    const double* B = g->B;
    const double V = g->V;
    const long n1 = M1 + 1, n2 = 2 * M2 + 1, n3 = 2 * M3 + 1;
    const long total = n1 * n2 * n3;
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (long start = 0; start < total; start += blockDim.x) {
        long lin = start + threadIdx.x;
        int keep = 0;
        double kx = 0, ky = 0, kz = 0, k2 = 0;
        if (lin < total) {
            int m1 = (int)(lin / (n2 * n3));
            int m2 = (int)((lin / n3) % n2) - M2;
            int m3 = (int)(lin % n3) - M3;
            bool half = (m1 > 0) || (m1 == 0 && m2 > 0) || (m1 == 0 && m2 == 0 && m3 > 0);
            if (half) {
                kx = m1 * B[0] + m2 * B[3] + m3 * B[6];
                ky = m1 * B[1] + m2 * B[4] + m3 * B[7];
                kz = m1 * B[2] + m2 * B[5] + m3 * B[8];
                k2 = kx * kx + ky * ky + kz * kz;
                keep = k2 <= kcut * kcut * (1.0 + 1e-12);
            }
        }
        // block-wide exclusive scan of keep
        unsigned bal = __ballot_sync(0xffffffffu, keep);
        int wpre = __popc(bal & ((1u << lane) - 1u));
        if (lane == 0) warp_sums[wid] = __popc(bal);
        __syncthreads();
        if (wid == 0) {
            int v = (lane < (int)(blockDim.x >> 5)) ? warp_sums[lane] : 0;
            int incl = v;
            for (int o = 1; o < 32; o <<= 1) {
                int t = __shfl_up_sync(0xffffffffu, incl, o);
                if (lane >= o) incl += t;
            }
            warp_sums[lane] = incl - v;   // exclusive
        }
        __syncthreads();
        if (keep) {
            int pos = base + warp_sums[wid] + wpre;
            double w = ke * (4.0 * kPi / V) * exp(-k2 / (4.0 * alpha * alpha)) / k2;
            kv[pos] = Vec4d{kx, ky, kz, sqrt(w)};
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) base += warp_sums[wid] + wpre + keep;
        __syncthreads();
    }
    if (threadIdx.x == 0) *count = base;
}

__global__ void k_frac_to_cart(const Geom* __restrict__ g, const double* __restrict__ frac, int N,
                               double* __restrict__ cart)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= N) return;
    const double* A = g->A;
    double f0 = frac[3 * i], f1 = frac[3 * i + 1], f2 = frac[3 * i + 2];
    for (int c = 0; c < 3; ++c) cart[3 * i + c] = f0 * A[c] + f1 * A[3 + c] + f2 * A[6 + c];
}

// X[i][t] = sqrt(w_t) cos(k_t . r_i), X[i][K + t] = sqrt(w_t) sin(k_t . r_i); zero
// padding for columns 2K .. ldx-1.
__global__ void k_struct_factor(const Vec4d* __restrict__ kv, int K, const double* __restrict__ cart, int N,
                                double* __restrict__ X, int ldx)
{
    long idx = (long)blockIdx.x * blockDim.x + threadIdx.x;
    long total = (long)N * ldx;
    for (; idx < total; idx += (long)gridDim.x * blockDim.x) {
        int i = (int)(idx / ldx);
        int t = (int)(idx % ldx);
        double v = 0.0;
        if (t < 2 * K) {
            int kk = t < K ? t : t - K;
            Vec4d k = kv[kk];
            double ph = k.x * cart[3 * i] + k.y * cart[3 * i + 1] + k.z * cart[3 * i + 2];
            double s, c;
            sincos(ph, &s, &c);
            v = k.w * (t < K ? c : s);
        }
        X[idx] = v;
    }
}

// J[i][j] = sum_t X[i][t] X[j][t] for 64x64 tiles (bi >= bj), 256 threads,
// 4x4 outputs per thread, K chunks of 16.
constexpr int SY_BM = 64, SY_BK = 16;

__global__ void __launch_bounds__(256) k_syrk_f64(const double* __restrict__ X, int N, int ldx,
                                                  double* __restrict__ J)
{
    // map blockIdx.x to (bi, bj), bi >= bj
    int t = blockIdx.x;
    int bi = (int)((sqrt(8.0 * t + 1.0) - 1.0) * 0.5);
    while ((bi + 1) * (bi + 2) / 2 <= t) ++bi;
    while (bi * (bi + 1) / 2 > t) --bi;
    int bj = t - bi * (bi + 1) / 2;
    const int i0 = bi * SY_BM, j0 = bj * SY_BM;

    __shared__ double As[SY_BK][SY_BM + 1];
    __shared__ double Bs[SY_BK][SY_BM + 1];
    const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
    double acc[4][4] = {};
    for (int k0 = 0; k0 < ldx; k0 += SY_BK) {
        for (int e = threadIdx.x; e < SY_BM * SY_BK; e += 256) {
            int r = e / SY_BK, c = e % SY_BK;
            int gi = i0 + r, gj = j0 + r;
            As[c][r] = gi < N ? X[(long)gi * ldx + k0 + c] : 0.0;
            Bs[c][r] = gj < N ? X[(long)gj * ldx + k0 + c] : 0.0;
        }
        __syncthreads();
#pragma unroll
        for (int k = 0; k < SY_BK; ++k) {
            double a[4], b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                a[u] = As[k][ty * 4 + u];
                b[u] = Bs[k][tx * 4 + u];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
                for (int v = 0; v < 4; ++v) acc[u][v] = fma(a[u], b[v], acc[u][v]);
        }
        __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
            int gi = i0 + ty * 4 + u, gj = j0 + tx * 4 + v;
            if (gi < N && gj < N) J[(long)gi * N + gj] = acc[u][v];
        }
}

// Real-space image sum for pairs i <= j, plus self and background; the
// reciprocal part is read from the lower triangle written by k_syrk_f64.
// Terms with alpha r >= 6 are skipped (erfc(6) = 2.2e-17).  The image list is
// first screened with an FP32 distance test whose cutoff carries a 1e-4
// relative margin (FP32 r^2 is within 1e-6 of FP64), so no image that the FP64
// test keeps is ever screened out; every kept term is evaluated in FP64.
constexpr double kRealCut = 6.0;
constexpr int kMaxImgF = 1024;

__global__ void __launch_bounds__(256) k_real_space(const Geom* __restrict__ g, const double* __restrict__ frac,
                                                    int N, const Vec4d* __restrict__ img, int nimg_total,
                                                    double alpha, double ke, double* __restrict__ J)
{
    __shared__ float4 imgf[kMaxImgF];
    if (blockIdx.x < blockIdx.y) return;   // tile strictly below the diagonal (uniform per block)
    const bool screen = nimg_total <= kMaxImgF;
    if (screen)
        for (int t = threadIdx.y * 16 + threadIdx.x; t < nimg_total; t += 256) {
            const Vec4d n = img[t];
            imgf[t] = make_float4((float)n.x, (float)n.y, (float)n.z, (float)n.w);
        }
    __syncthreads();
    const int i = blockIdx.y * 16 + threadIdx.y;
    const int j = blockIdx.x * 16 + threadIdx.x;
    if (i >= N || j >= N || i > j) return;
    const double* A = g->A;
    double df[3];
    for (int c = 0; c < 3; ++c) {
        double x = frac[3 * j + c] - frac[3 * i + c];
        df[c] = x - floor(x + 0.5);
    }
    double d[3];
    for (int c = 0; c < 3; ++c) d[c] = df[0] * A[c] + df[1] * A[3 + c] + df[2] * A[6 + c];
    const double rc2 = kRealCut * kRealCut / (alpha * alpha);
    const float rc2f = (float)(rc2 * (1.0 + 1e-4));
    const float dx = (float)d[0], dy = (float)d[1], dz = (float)d[2];
    double real = 0.0;
    for (int t = 0; t < nimg_total; ++t) {
        if (screen) {
            const float4 nf = imgf[t];
            const float fx = dx + nf.x, fy = dy + nf.y, fz = dz + nf.z;
            if (fx * fx + fy * fy + fz * fz >= rc2f) continue;
        }
        const Vec4d n = img[t];
        if (i == j && n.w != 0.0) continue;      // n = 0 term of the self pair
        double rx = d[0] + n.x, ry = d[1] + n.y, rz = d[2] + n.z;
        double r2 = rx * rx + ry * ry + rz * rz;
        if (r2 >= rc2) continue;
        double r = sqrt(r2);
        real += erfc(alpha * r) / r;
    }
    const double V = g->V;
    double self = (i == j) ? -2.0 * alpha / sqrt(kPi) : 0.0;
    double bg = -kPi / (V * alpha * alpha);
    double v = 0.5 * ke * (real + self + bg) + J[(long)j * N + i];
    J[(long)i * N + j] = v;
    J[(long)j * N + i] = v;
}

// Image translations n1 a1 + n2 a2 + n3 a3 for |n_a| <= nimg[a]; w = 1 marks n = 0.
__global__ void k_images(const Geom* __restrict__ g, int n1, int n2, int n3, Vec4d* __restrict__ img)
{
    int t = blockIdx.x * blockDim.x + threadIdx.x;
    int tot = (2 * n1 + 1) * (2 * n2 + 1) * (2 * n3 + 1);
    if (t >= tot) return;
    int a = t / ((2 * n2 + 1) * (2 * n3 + 1)) - n1;
    int b = (t / (2 * n3 + 1)) % (2 * n2 + 1) - n2;
    int c = t % (2 * n3 + 1) - n3;
    const double* A = g->A;
    double x = a * A[0] + b * A[3] + c * A[6];
    double y = a * A[1] + b * A[4] + c * A[7];
    double z = a * A[2] + b * A[5] + c * A[8];
    img[t] = Vec4d{x, y, z, (a == 0 && b == 0 && c == 0) ? 1.0 : 0.0};
}

}  // namespace

extern "C" goac_status goac_build_ewald(goac_ctx* ctx, const double* lattice_host, const double* frac_dev, int32_t N,
                                        double alpha, const int32_t* nimg_host, double kcut, double ke, double* J_dev)
{
    if (!ctx || !lattice_host || !frac_dev || !nimg_host || !J_dev || N <= 0)
        return goac::fail(GOAC_ERR_INVALID_ARG, "goac_build_ewald: null pointer or N <= 0");
    if (!(alpha > 0.0) || !(kcut >= 0.0) || !(ke > 0.0))
        return goac::fail(GOAC_ERR_INVALID_ARG, "goac_build_ewald: alpha, ke must be > 0 and kcut >= 0");
    for (int a = 0; a < 3; ++a)
        if (nimg_host[a] < 0 || nimg_host[a] > 64)
            return goac::fail(GOAC_ERR_INVALID_ARG, "goac_build_ewald: nimg out of range [0, 64]");
    GOAC_CUDA(cudaSetDevice(ctx->device));
    cudaStream_t st = ctx->stream;

    // index-box bounds |m_a| <= kcut |a_a| / (2 pi) (+1 margin): loop bounds only
    int M[3];
    for (int d = 0; d < 3; ++d) {
        double al = sqrt(lattice_host[3 * d] * lattice_host[3 * d] + lattice_host[3 * d + 1] * lattice_host[3 * d + 1] +
                         lattice_host[3 * d + 2] * lattice_host[3 * d + 2]);
        M[d] = (int)floor(kcut * al / (2.0 * kPi)) + 1;
    }
    long box = (long)(M[0] + 1) * (2 * M[1] + 1) * (2 * M[2] + 1);
    if (box > (1L << 24)) return goac::fail(GOAC_ERR_INVALID_ARG, "goac_build_ewald: kcut too large");
    const int nimg_total = (2 * nimg_host[0] + 1) * (2 * nimg_host[1] + 1) * (2 * nimg_host[2] + 1);

    double* dA = nullptr;
    Geom* dG = nullptr;
    Vec4d* dK = nullptr;
    int* dCount = nullptr;
    double* dCart = nullptr;
    Vec4d* dImg = nullptr;
    double* dX = nullptr;
    goac_status rc = GOAC_OK;
    int K = 0;
    auto cleanup = [&]() {
        cudaFree(dA);
        cudaFree(dG);
        cudaFree(dK);
        cudaFree(dCount);
        cudaFree(dCart);
        cudaFree(dImg);
        cudaFree(dX);
    };
#define TRY(call)                                          \
    do {                                                   \
        cudaError_t e__ = (call);                          \
        if (e__ != cudaSuccess) {                          \
            rc = goac::cuda_fail(e__, #call);              \
            cleanup();                                     \
            return rc;                                     \
        }                                                  \
    } while (0)
    TRY(cudaMalloc(&dA, 9 * sizeof(double)));
    TRY(cudaMalloc(&dG, sizeof(Geom)));
    TRY(cudaMalloc(&dK, sizeof(Vec4d) * (box + 1)));
    TRY(cudaMalloc(&dCount, sizeof(int)));
    TRY(cudaMalloc(&dCart, sizeof(double) * 3 * N));
    TRY(cudaMalloc(&dImg, sizeof(Vec4d) * nimg_total));
    TRY(cudaMemcpyAsync(dA, lattice_host, 9 * sizeof(double), cudaMemcpyHostToDevice, st));
    goac::launch(k_geometry, 1, 32, 0, st, dA, dG);
    goac::launch(k_kvectors, 1, 1024, 0, st, dG, M[0], M[1], M[2], kcut, alpha, ke, dK, dCount);
    goac::launch(k_frac_to_cart, (N + 255) / 256, 256, 0, st, dG, frac_dev, N, dCart);
    goac::launch(k_images, (nimg_total + 255) / 256, 256, 0, st, dG, nimg_host[0], nimg_host[1], nimg_host[2], dImg);
    TRY(cudaGetLastError());
    TRY(cudaMemcpyAsync(&K, dCount, sizeof(int), cudaMemcpyDeviceToHost, st));
    TRY(cudaStreamSynchronize(st));

    const int ldx = ((2 * K + 15) / 16) * 16 + (K == 0 ? 16 : 0);
    TRY(cudaMalloc(&dX, sizeof(double) * (size_t)N * ldx));
    {
        long total = (long)N * ldx;
        int blocks = (int)((total + 255) / 256);
        if (blocks > 65535 * 16) blocks = 65535 * 16;
        goac::launch(k_struct_factor, blocks, 256, 0, st, dK, K, dCart, N, dX, ldx);
    }
    {
        int nb = (N + SY_BM - 1) / SY_BM;
        long ntiles = (long)nb * (nb + 1) / 2;
        goac::KTimer kt(ctx, goac::KID_EWALD_SYRK, st);
        goac::launch(k_syrk_f64, (unsigned)ntiles, 256, 0, st, dX, N, ldx, J_dev);
    }
    {
        dim3 grid((N + 15) / 16, (N + 15) / 16), block(16, 16);
        goac::KTimer kt(ctx, goac::KID_EWALD_REAL, st);
        goac::launch(k_real_space, grid, block, 0, st, dG, frac_dev, N, dImg, nimg_total, alpha, ke, J_dev);
    }
    TRY(cudaGetLastError());
    TRY(cudaStreamSynchronize(st));
#undef TRY
    cleanup();
    return GOAC_OK;
}
