// estimate.cu -- reverberation-parameter estimation from the SH energy IR
// (Section 4.2), in FP64.  One block per source, one warp per band; lane l owns a
// contiguous run of bins.
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

__global__ void k_estimate(EstimateWork w)
{
    __shared__ int first_nz[MAXB];
    const int s = blockIdx.x;
    const int b = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int B = w.B, K = w.K, T = w.T;
    const double sq4pi = sqrt(4.0 * 3.14159265358979323846);
    const float *h0 = w.H + (((size_t)s * B + b) * K + 0) * T;
    const int per = (T + 31) / 32;
    const int j0 = min(T, lane * per), j1 = min(T, j0 + per);

    // chunk total and first non-zero bin
    double tot = 0.0;
    int fnz = T;
    for (int j = j0; j < j1; ++j) {
        const double I = sq4pi * (double)h0[j];
        tot += I;
        if (I > 0.0 && fnz == T) fnz = j;
    }
    fnz = wmin_i(fnz);
    if (lane == 0) first_nz[b] = fnz;
    // tail[l] = sum of the chunk totals of lanes > l (suffix scan)
    double incl = tot;
    for (int o = 1; o < 32; o <<= 1) {
        const double y = __shfl_down_sync(FULL, incl, o);
        if (lane + o < 32) incl += y;
    }
    const double tail = incl - tot;
    const double E0 = __shfl_sync(FULL, incl, 0);
    const double itot = wsum(tot);

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
        double suf = tail;
        for (int j = j1 - 1; j >= j0; --j) {
            suf += sq4pi * (double)h0[j];
            const double Lj = suf > 0.0 ? 10.0 * log10(suf / E0) : -INFINITY;
#pragma unroll
            for (int r = 0; r < 3; ++r) {
                above_hi[r] += Lj > HI[r];
                above_lo[r] += Lj >= LO[r];
            }
        }
    }
#pragma unroll
    for (int r = 0; r < 3; ++r) {
        above_hi[r] = wsum_i(above_hi[r]);
        above_lo[r] = wsum_i(above_lo[r]);
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
            sy = wsum(sy);
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
            sxx = wsum(sxx);
            sxy = wsum(sxy);
            syy = wsum(syy);
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
        xs[kk] = wsum(a);
    }
    __syncthreads();
    int first = T;
    for (int bb = 0; bb < B; ++bb) first = min(first, first_nz[bb]);

    if (lane == 0) {
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
        o.predelay_s = first < T ? (double)first / w.rate : NAN;
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

}  // namespace

void launch_estimate(const EstimateWork &w, cudaStream_t st)
{
    if (w.S <= 0) return;
    k_estimate<<<w.S, 32 * w.B, 0, st>>>(w);
}

}  // namespace rp
