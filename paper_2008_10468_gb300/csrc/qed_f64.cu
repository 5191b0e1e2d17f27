// GB300 (sm_103a) binary64 synchrotron functions: the C ABI entry
// qed_synchrotron_F1F2_f64 of include/qed.h.
//
// F(x) = x int_x^inf K_{5/3}(t) dt and G(x) = x K_{2/3}(x) (Sec. 3.2.1) to
// ~1e-15 relative error, the double-precision accuracy level of Table 1, from
// the tables of fit_synchrotron64.py: per piece [1, 1.25), [1.25, 1.5), [1.5, 2)
// of m in x = m 2^k,
//   F = 2^{k/3} exp(-lam_k x) sum_j c_j u^j,  u = (m - centre) / halfwidth in [-1, 1)
// (u exact: dyadic centres and half-widths), and below 2^KMIN the small-x
// series F = x^{1/3} sum_j a_j x^{2j/3}.
// No difference of two large terms is formed, so the binary64 evaluation
// keeps the fit's accuracy; arguments from 2^(KMAX+1) on give 0 (F, G < 1e-220).
#include <cstdint>

#include "qed.h"
#include "synchro_coeffs64.h"

namespace {

constexpr int kCoef64 = 2 * (QED_SYN64_DEG + 1);
constexpr int kPieceStride64 = 72;   // pieces padded (NPIECE <= 72)
static_assert(QED_SYN64_NPIECE <= kPieceStride64, "piece stride");
constexpr int kThreads64 = 256;

struct Syn64Table {
    double c[kCoef64][kPieceStride64];   // [coefficient][piece]: lanes of a warp in
                                         // different pieces read different banks
    double scale[kPieceStride64];        // 2^{k/3} of the piece's octave
    double small[2][QED_SYN64_SMALL_DEG + 1];
};

__device__ void stage_syn64(Syn64Table& T) {
    for (int i = threadIdx.x; i < kCoef64 * kPieceStride64; i += blockDim.x) {
        const int j = i / kPieceStride64, p = i % kPieceStride64;
        T.c[j][p] = p < QED_SYN64_NPIECE ? qed_syn64_table[p][j] : 0.0;
    }
    for (int p = threadIdx.x; p < kPieceStride64; p += blockDim.x) {
        const int k = QED_SYN64_KMIN + p / 3;
        T.scale[p] = exp2((double)k / 3.0);
    }
    for (int i = threadIdx.x; i < 2 * (QED_SYN64_SMALL_DEG + 1); i += blockDim.x)
        T.small[i / (QED_SYN64_SMALL_DEG + 1)][i % (QED_SYN64_SMALL_DEG + 1)] =
            qed_syn64_small[i / (QED_SYN64_SMALL_DEG + 1)][i % (QED_SYN64_SMALL_DEG + 1)];
}

__device__ __forceinline__ void syn64(const Syn64Table& T, double x, double& F, double& G) {
    const double x_max = (double)(1ll << (QED_SYN64_KMAX + 1));
    if (!(x > 0.0) || !(x < x_max)) {   // also NaN
        F = G = 0.0;
        return;
    }
    const long long bits = __double_as_longlong(x);
    const int e = (int)((bits >> 52) & 0x7FF);
    const int k = e - 1023;
    if (e == 0 || k < QED_SYN64_KMIN) {   // small-x series (subnormals included)
        const double r = cbrt(x);
        const double v = r * r;
        double pf = T.small[0][QED_SYN64_SMALL_DEG], pg = T.small[1][QED_SYN64_SMALL_DEG];
#pragma unroll
        for (int j = QED_SYN64_SMALL_DEG - 1; j >= 0; --j) {
            pf = fma(pf, v, T.small[0][j]);
            pg = fma(pg, v, T.small[1][j]);
        }
        F = r * pf;
        G = r * pg;
        return;
    }
    const double m = __longlong_as_double((bits & 0x000FFFFFFFFFFFFFll) | 0x3FF0000000000000ll);
    const int part = m < 1.25 ? 0 : (m < 1.5 ? 1 : 2);
    const double centre = part == 0 ? 1.125 : (part == 1 ? 1.375 : 1.75);
    const double inv_half = part == 2 ? 4.0 : 8.0;
    const double u = (m - centre) * inv_half;
    const int p = 3 * (k - QED_SYN64_KMIN) + part;
    double pf = T.c[QED_SYN64_DEG][p], pg = T.c[2 * QED_SYN64_DEG + 1][p];
#pragma unroll
    for (int j = QED_SYN64_DEG - 1; j >= 0; --j) {
        pf = fma(pf, u, T.c[j][p]);
        pg = fma(pg, u, T.c[QED_SYN64_DEG + 1 + j][p]);
    }
    double s = T.scale[p];
    if (k >= QED_SYN64_LAMBDA_FROM) s *= exp(-x);
    F = s * pf;
    G = s * pg;
}

__global__ void __launch_bounds__(kThreads64) k_sweep64(const double* __restrict__ y,
                                                        double* __restrict__ F1,
                                                        double* __restrict__ F2, long long n) {
    __shared__ Syn64Table T;
    stage_syn64(T);
    __syncthreads();
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        double a, b;
        syn64(T, __ldcs(y + i), a, b);
        if (F1) __stcs(F1 + i, a);
        if (F2) __stcs(F2 + i, b);
    }
}

}  // namespace

extern "C" qed_status qed_synchrotron_F1F2_f64(const double* y, double* F1, double* F2,
                                                int64_t n, void* stream) {
    if (n < 0 || (n > 0 && (!y || (!F1 && !F2)))) return QED_ERR_ARG;
    if (n == 0) return QED_OK;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return QED_ERR_CUDA;
    const long long blocks = ((long long)n + kThreads64 - 1) / kThreads64;
    const int grid = (int)(blocks < (long long)sms * 8 ? blocks : (long long)sms * 8);
    k_sweep64<<<grid, kThreads64, 0, (cudaStream_t)stream>>>(y, F1, F2, (long long)n);
    return cudaGetLastError() == cudaSuccess ? QED_OK : QED_ERR_CUDA;
}
