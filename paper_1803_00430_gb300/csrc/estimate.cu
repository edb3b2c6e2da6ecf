// estimate.cu -- reverberation-parameter estimation from the SH energy IR
// (Section 4.2), in FP64.  One block per (source, band); thread l owns a contiguous
// run of bins.
//
//   I_b(t)      = sqrt(4 pi) X_{b,00}(t)                    (Y_00 = 1/sqrt(4 pi))
//   E_b(t)      = sum_{t' >= t} I_b(t')                     backward integration
//   L_b(t)      = 10 log10(E_b(t) / E_b(0))
//   fit window  = T30 (-5..-35 dB), else T20 (-5..-25 dB), else T10 (0..-10 dB),
//                 usable when it spans >= 3 bins and the curve falls below its floor
//   RT60        = -60 / slope of the least-squares line of L on bin start time
//   I_total     = sum_t I_b(t);  g_reverb = sqrt(I_total / (RT60 / (6 ln 10)))
//                 (Eq. reverb_gain with the reverberator's total intensity)
//   DRR         = 10 log10(E_direct / I_total)
//   predelay    = first bin non-zero in any band, / rate
//   X-bar_lm    = sum_t X_{b,lm}(t) / I_total              (Section 4.1)
//   smoothing   = alpha * RT60 + (1 - alpha) * previous, alpha = 1 - exp(-dt / tau)
//
// The window ends come from counting the bins whose level is above each threshold
// (the decay curve never increases).  A level is compared through the energy ratio
// E(t) / E(0) against 10^(threshold / 10); only a ratio within a relative 1e-9 of a
// threshold, where rounding of the logarithm could matter, takes the logarithm, so
// every decision equals the one on L_b(t) and most bins need no FP64 logarithm.
#include <cmath>

#include "internal.cuh"

namespace rp {
namespace {

__device__ __forceinline__ double wsum(double v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

__device__ __forceinline__ int wsum_i(int v)
{
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
    return v;
}

__device__ __forceinline__ int wmin_i(int v)
{
    for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(FULL, v, o));
    return v;
}

constexpr int EST_THREADS = 128;

// block-wide sums (all threads get the result); `sh` holds EST_THREADS / 32 doubles
__device__ __forceinline__ double bsum(double v, double *sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = wsum(v);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = 0.0;
    for (int i = 0; i < EST_THREADS / 32; ++i) t += sh[i];
    return t;
}

__device__ __forceinline__ int bsum_i(int v, int *sh)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    v = wsum_i(v);
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    int t = 0;
    for (int i = 0; i < EST_THREADS / 32; ++i) t += sh[i];
    return t;
}

// whether 10 log10(ratio) > c (strict) or >= c, with thr = 10^(c / 10)
__device__ __forceinline__ bool level_above(double ratio, double c, double thr, bool strict)
{
    if (ratio > thr * (1.0 + 1e-9)) return true;
    if (ratio < thr * (1.0 - 1e-9)) return false;
    const double L = ratio > 0.0 ? 10.0 * log10(ratio) : -INFINITY;
    return strict ? L > c : L >= c;
}

__global__ void __launch_bounds__(EST_THREADS) k_estimate(EstimateWork w)
{
    __shared__ double shd[EST_THREADS / 32];
    __shared__ int shi[EST_THREADS / 32];
    __shared__ double scan[EST_THREADS];
    const int s = blockIdx.x / w.B, b = blockIdx.x % w.B;
    const int t = threadIdx.x;
    const int B = w.B, K = w.K, T = w.T;
    const double sq4pi = sqrt(4.0 * 3.14159265358979323846);
    const float *h0 = w.H + (((size_t)s * B + b) * K + 0) * T;
    const int per = (T + EST_THREADS - 1) / EST_THREADS;
    const int j0 = min(T, t * per), j1 = min(T, j0 + per);
    // chunk total and first non-zero bin
    double tot = 0.0;
    int fnz = T;
    for (int j = j0; j < j1; ++j) {
        const double I = sq4pi * (double)h0[j];
        tot += I;
        if (I > 0.0 && fnz == T) fnz = j;
    }
    // tail = sum of the chunk totals of threads > t (inclusive suffix scan)
    scan[t] = tot;
    __syncthreads();
    for (int o = 1; o < EST_THREADS; o <<= 1) {
        const double y = t + o < EST_THREADS ? scan[t + o] : 0.0;
        __syncthreads();
        scan[t] += y;
        __syncthreads();
    }
    const double tail = scan[t] - tot;
    const double E0 = scan[0];
    const double itot = E0;
    int first = fnz;
    {
        first = wmin_i(first);
        __syncthreads();
        if ((t & 31) == 0) shi[t >> 5] = first;
        __syncthreads();
        for (int i = 0; i < EST_THREADS / 32; ++i) first = min(first, shi[i]);
        __syncthreads();
    }
    // level of the last bin decides whether a floor is reached
    double Llast = -INFINITY;
    {
        const double Il = sq4pi * (double)h0[T - 1];
        if (E0 > 0.0 && Il > 0.0) Llast = 10.0 * log10(Il / E0);
    }
    static const double HI[3] = {-5.0, -5.0, 0.0};
    static const double LO[3] = {-35.0, -25.0, -10.0};
    int above_hi[3] = {0, 0, 0}, above_lo[3] = {0, 0, 0};
    if (E0 > 0.0) {
        double thi[3], tlo[3];
#pragma unroll
        for (int r = 0; r < 3; ++r) {
            thi[r] = pow(10.0, HI[r] / 10.0);
            tlo[r] = pow(10.0, LO[r] / 10.0);
        }
        double suf = tail;
        for (int j = j1 - 1; j >= j0; --j) {
            suf += sq4pi * (double)h0[j];
            const double ratio = suf / E0;
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                above_hi[r] += level_above(ratio, HI[r], thi[r], true);
                above_lo[r] += level_above(ratio, LO[r], tlo[r], false);
            }
        }
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        above_hi[r] = bsum_i(above_hi[r], shi);
        above_lo[r] = bsum_i(above_lo[r], shi);
    }
    double rt = NAN, slope = NAN, icpt = NAN, r2 = NAN, fhi = 0.0, flo = 0.0;
    int kind = 0, nfit = 0, fa = -1, fz = -1;
    if (E0 > 0.0) {
        for (int r = 0; r < 3 && kind == 0; ++r) {
            // the decay curve is non-increasing: the window is [a, z]
            const int a = above_hi[r], z = above_lo[r] - 1;
            const int n = z - a + 1;
            const bool reached = Llast < LO[r];
            if (n < 3 || !reached) continue;
            // mean level over the window
            double sy = 0.0;
            {
                double suf = tail;
                for (int j = j1 - 1; j >= j0; --j) {
                    suf += sq4pi * (double)h0[j];
                    if (j >= a && j <= z) sy += 10.0 * log10(suf / E0);
                }
            }
            sy = bsum(sy, shd);
            const double my = sy / n;
            const double mx = 0.5 * (double)(a + z) / w.rate;
            double sxx = 0.0, sxy = 0.0, syy = 0.0;
            {
                double suf = tail;
                for (int j = j1 - 1; j >= j0; --j) {
                    suf += sq4pi * (double)h0[j];
                    if (j >= a && j <= z) {
                        const double dx = (double)j / w.rate - mx;
                        const double dy = 10.0 * log10(suf / E0) - my;
                        sxx += dx * dx;
                        sxy += dx * dy;
                        syy += dy * dy;
                    }
                }
            }
            sxx = bsum(sxx, shd);
            sxy = bsum(sxy, shd);
            syy = bsum(syy, shd);
            const double sl = sxy / sxx;
            if (!(sl < 0.0)) continue;
            slope = sl;
            icpt = my - sl * mx;
            r2 = syy > 0.0 ? (sxy * sxy) / (sxx * syy) : 1.0;
            rt = -60.0 / sl;
            kind = r + 1;
            nfit = n;
            fa = a;
            fz = z;
            fhi = HI[r];
            flo = LO[r];
        }
    }
    // weighted average directivity: sum_t X_k(t) / I_total
    double xs[MAXK];
#pragma unroll
    for (int kk = 0; kk < MAXK; ++kk) xs[kk] = 0.0;
    for (int kk = 0; kk < K; ++kk) {
        const float *hk = w.H + (((size_t)s * B + b) * K + kk) * T;
        double a = 0.0;
        for (int j = j0; j < j1; ++j) a += (double)hk[j];
        xs[kk] = bsum(a, shd);
    }
    if (t == 0) {
        rp_reverb_params o;
        o.rt60_raw = rt;
        o.fit_hi_db = fhi;
        o.fit_lo_db = flo;
        o.fit_r2 = r2;
        o.slope_db_per_s = slope;
        o.intercept_db = icpt;
        o.i_total = itot;
        o.g_reverb = kind > 0 ? sqrt(itot / (rt / (6.0 * log(10.0)))) : NAN;
        const double ed = (w.direct && w.direct[s].visible) ? (double)w.direct[s].energy : 0.0;
        o.e_direct = ed;
        if (ed > 0.0 && itot > 0.0) o.drr_db = 10.0 * log10(ed / itot);
        else if (ed > 0.0) o.drr_db = INFINITY;
        else if (itot > 0.0) o.drr_db = -INFINITY;
        else o.drr_db = NAN;
        // this band's first non-zero bin; k_predelay turns it into the source's predelay
        o.predelay_s = (double)first;
        o.range_kind = kind;
        o.n_fit = nfit;
        o.fit_j0 = fa;
        o.fit_j1 = fz;
        for (int kk = 0; kk < MAXK; ++kk) o.xbar[kk] = (kk < K && itot > 0.0) ? xs[kk] / itot : (kk < K ? NAN : 0.0);
        double sm = rt;
        if (w.state) {
            const double prev = w.state[(size_t)s * B + b];
            const double alpha = w.tau > 0.0 ? 1.0 - exp(-w.dt / w.tau) : 1.0;
            if (isnan(prev)) sm = rt;
            else if (isnan(rt)) sm = prev;
            else sm = alpha * rt + (1.0 - alpha) * prev;
            w.state[(size_t)s * B + b] = sm;
        }
        o.rt60_smoothed = sm;
        w.out[(size_t)s * B + b] = o;
    }
}

// predelay of every source: its earliest non-zero bin over the bands (Section 4.2,
// "for all frequency bands"), from the per-band first bins k_estimate left in
// predelay_s
__global__ void k_predelay(EstimateWork w)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= w.S) return;
    rp_reverb_params *o = w.out + (size_t)s * w.B;
    double first = (double)w.T;
    for (int b = 0; b < w.B; ++b) first = fmin(first, o[b].predelay_s);
    const double p = first < (double)w.T ? first / w.rate : NAN;
    for (int b = 0; b < w.B; ++b) o[b].predelay_s = p;
}

}  // namespace

void launch_estimate(const EstimateWork &w, cudaStream_t st)
{
    if (w.S <= 0) return;
    k_estimate<<<w.S * w.B, EST_THREADS, 0, st>>>(w);
    k_predelay<<<(w.S + 127) / 128, 128, 0, st>>>(w);
}

}  // namespace rp
