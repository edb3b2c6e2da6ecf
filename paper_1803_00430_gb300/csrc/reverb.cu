// reverb.cu -- the reverberator's parameters from the estimated ones (Section 4.1
// "Sound Rendering" and Section 4.2 "Reflection Density"), per source:
//   comb delays    N_comb feedback delays drawn from a Gaussian about r_free / c with
//                  sigma = (r_free / c) / 3, drawn again only when r_free / c has moved by
//                  more than 2 sigma from the mean they were drawn for (Philox key =
//                  seed, counter (source, comb, draw generation, 3); Box-Muller);
//   comb gains     g_comb = 10^(-3 t_comb / RT60) per band (comb feedback gain equation);
//   input          the dominant direction of the early IR directivity at t_comb past
//                  the first non-zero bin, normalize(-X_11, -X_1-1, X_10), and the comb's
//                  SH input gains Y_lm(direction) / N_comb;
//   rotations      a random rotation per comb, each angle in [90, 270] degrees about x,
//                  y and z (Philox counter (source, comb, 0, 2)), and its SH rotation
//                  matrix J by the recurrence of Ivanic and Ruedenberg (1996, with the
//                  1998 erratum), built up degree by degree from the 3 x 3 rotation;
//   loudness       per band, the directional loudness matrix D from the average
//                  directivity xbar: its direction density sampled on a product Gauss
//                  rule (the paper's spherical t-design) gives an amplitude gain per
//                  direction, and D = sum_j w_j a(x_j) Y(x_j) Y(x_j)^T.
#include <cmath>

#include "handles.cuh"

using namespace rp;

namespace rp {
namespace {

constexpr int N_COMB = RP_N_COMB;
constexpr int MAXQ = 8;  // Gauss-Legendre nodes in cos(theta) (2n + 2 for SH order n <= 3)

struct SphereRule {
    double z[MAXQ], w[MAXQ];
    int nt, nphi;
};

__device__ __forceinline__ double u01d(uint32_t x) { return (double)(x >> 8) * (1.0 / 16777216.0); }

// SH rotation by recurrence.  Rl[l][l + m][l + m'] in the real SH without the
// Condon-Shortley phase (degree 1 in the order y, z, x); the library's basis carries the
// phase (-1)^m, applied at the end.
struct ShRot {
    double r[4][7][7];
    __host__ __device__ double get(int l, int m, int mp) const { return r[l][l + m][l + mp]; }
    __host__ __device__ double P(int i, int a, int b, int l) const
    {
        const double ri1 = get(1, i, 1), rim1 = get(1, i, -1), ri0 = get(1, i, 0);
        if (b == l) return ri1 * get(l - 1, a, l - 1) - rim1 * get(l - 1, a, -l + 1);
        if (b == -l) return ri1 * get(l - 1, a, -l + 1) + rim1 * get(l - 1, a, l - 1);
        return ri0 * get(l - 1, a, b);
    }
    __host__ __device__ void build(const double R[3][3], int order)
    {
        r[0][0][0] = 1.0;
        const int ax[3] = {1, 2, 0};  // degree-1 index m + 1 -> axis y, z, x
        for (int m = -1; m <= 1; ++m)
            for (int mp = -1; mp <= 1; ++mp) r[1][m + 1][mp + 1] = R[ax[m + 1]][ax[mp + 1]];
        for (int l = 2; l <= order; ++l) {
            for (int m = -l; m <= l; ++m) {
                for (int mp = -l; mp <= l; ++mp) {
                    const double d = (mp > -l && mp < l) ? (double)((l + mp) * (l - mp)) : (double)(2 * l * (2 * l - 1));
                    const int am = m < 0 ? -m : m;
                    const double dm0 = m == 0 ? 1.0 : 0.0;
                    const double u = sqrt((double)((l + m) * (l - m)) / d);
                    const double v = 0.5 * sqrt((1.0 + dm0) * (double)((l + am - 1) * (l + am)) / d) * (1.0 - 2.0 * dm0);
                    const double w = -0.5 * sqrt((double)((l - am - 1) * (l - am)) / d) * (1.0 - dm0);
                    double val = 0.0;
                    if (u != 0.0) val += u * P(0, m, mp, l);
                    if (v != 0.0) {
                        double V;
                        if (m == 0) V = P(1, 1, mp, l) + P(-1, -1, mp, l);
                        else if (m > 0) V = P(1, m - 1, mp, l) * sqrt(m == 1 ? 2.0 : 1.0) - (m == 1 ? 0.0 : P(-1, -m + 1, mp, l));
                        else V = (m == -1 ? 0.0 : P(1, m + 1, mp, l)) + P(-1, -m - 1, mp, l) * sqrt(m == -1 ? 2.0 : 1.0);
                        val += v * V;
                    }
                    if (w != 0.0) {
                        const double W = m > 0 ? P(1, m + 1, mp, l) + P(-1, -m - 1, mp, l)
                                               : P(1, m - 1, mp, l) - P(-1, -m + 1, mp, l);
                        val += w * W;
                    }
                    r[l][l + m][l + mp] = val;
                }
            }
        }
    }
};

// one warp per source
__global__ void __launch_bounds__(32) k_reverb_config(const float *__restrict__ H, const rp_reverb_params *prm, int S,
                                                      int B, int K, int T, double rate, double mean, unsigned long long seed,
                                                      SphereRule rule, rp_reverberator *rev)
{
    const int s = blockIdx.x;
    if (s >= S) return;
    const int lane = threadIdx.x;
    const int order = K >= 16 ? 3 : (K >= 9 ? 2 : (K >= 4 ? 1 : 0));
    const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
    rp_reverberator &R = rev[s];
    // the draw: kept unless r_free / c moved by more than 2 sigma of the mean it was drawn for
    const uint32_t gen0 = R.generation;
    const double mu0 = R.mean_delay_s;
    const bool redraw = gen0 == 0u || fabs(mean - mu0) > 2.0 * mu0 / 3.0;
    const uint32_t gen = redraw ? gen0 + 1u : gen0;
    const double mu = redraw ? mean : mu0;
    __syncwarp();
    // first non-zero bin of the omnidirectional IR over bands
    int first = T;
    for (int j = lane; j < T; j += 32) {
        float I = 0.f;
        for (int b = 0; b < B; ++b) I += H[(((size_t)s * B + b) * K) * T + j];
        if (I > 0.f) {
            first = j;
            break;
        }
    }
    for (int o = 16; o > 0; o >>= 1) first = min(first, __shfl_xor_sync(0xffffffffu, first, o));
    if (lane < N_COMB) {
        const int i = lane;
        // delay: Box-Muller from the (0, 1] and [0, 1) uniforms of one Philox block
        const U4 r = philox4x32_10((uint32_t)s, (uint32_t)i, gen, 3u, k0, k1);
        const double u1 = (double)((r.x >> 8) + 1u) * (1.0 / 16777216.0), u2 = u01d(r.y);
        const double t = fmax(mu + mu / 3.0 * sqrt(-2.0 * log(u1)) * cos(2.0 * 3.141592653589793 * u2), mu / 10.0);
        R.t_comb[i] = t;
        for (int b = 0; b < RP_MAX_BANDS; ++b) {
            const double rt = b < B ? prm[(size_t)s * B + b].rt60_smoothed : 0.0;
            R.g_comb[i][b] = (b < B && rt > 0.0) ? exp(-3.0 * t / rt * 2.302585092994046) : 0.0;
        }
        // input direction from the band-summed first-order directivity at first + t
        double dir[3] = {0.0, 0.0, 1.0};
        if (first < T && K >= 4) {
            const double x = fmin((first / rate + t) * rate, (double)T - 1.0);
            const int j0 = (int)floor(x), j1 = min(j0 + 1, T - 1);
            const double f = x - j0;
            double v[3] = {0.0, 0.0, 0.0};
            for (int b = 0; b < B; ++b)
                for (int q = 0; q < 3; ++q) {
                    const float *h = H + (((size_t)s * B + b) * K + 1 + q) * T;
                    v[q] += (1.0 - f) * h[j0] + f * h[j1];
                }
            const double d[3] = {-v[2], -v[0], v[1]};
            const double n = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
            if (n > 0.0)
                for (int q = 0; q < 3; ++q) dir[q] = d[q] / n;
        }
        float Y[MAXK];
        sh_eval(order, (float)dir[0], (float)dir[1], (float)dir[2], Y);
        for (int q = 0; q < 3; ++q) R.dir[i][q] = dir[q];
        for (int kk = 0; kk < RP_MAX_SH; ++kk) R.comb_in[i][kk] = kk < K ? Y[kk] / (float)N_COMB : 0.f;
        // rotation: Rz(gamma) Ry(beta) Rx(alpha), angles in [pi/2, 3pi/2)
        const U4 ra = philox4x32_10((uint32_t)s, (uint32_t)i, 0u, 2u, k0, k1);
        const double a = 3.141592653589793 * (0.5 + u01d(ra.x)), be = 3.141592653589793 * (0.5 + u01d(ra.y)),
                     g = 3.141592653589793 * (0.5 + u01d(ra.z));
        const double ca = cos(a), sa = sin(a), cb = cos(be), sb = sin(be), cg = cos(g), sg = sin(g);
        const double Rm[3][3] = {{cg * cb, cg * sb * sa - sg * ca, cg * sb * ca + sg * sa},
                                 {sg * cb, sg * sb * sa + cg * ca, sg * sb * ca - cg * sa},
                                 {-sb, cb * sa, cb * ca}};
        for (int p = 0; p < 3; ++p)
            for (int q = 0; q < 3; ++q) R.rot[i][p][q] = (float)Rm[p][q];
        ShRot sr;
        sr.build(Rm, order);
        for (int k = 0; k < RP_MAX_SH; ++k)
            for (int kp = 0; kp < RP_MAX_SH; ++kp) R.J[i][k][kp] = 0.f;
        for (int l = 0; l <= order; ++l)
            for (int m = -l; m <= l; ++m)
                for (int mp = -l; mp <= l; ++mp) {
                    const double sgn = (((m < 0 ? -m : m) + (mp < 0 ? -mp : mp)) & 1) ? -1.0 : 1.0;  // (-1)^(m + m')
                    R.J[i][l * l + l + m][l * l + l + mp] = (float)(sgn * sr.get(l, m, mp));
                }
    }
    // directional loudness, one band per lane
    if (lane < RP_MAX_BANDS) {
        const int b = lane;
        double D[RP_MAX_SH * (RP_MAX_SH + 1) / 2];
        for (int q = 0; q < RP_MAX_SH * (RP_MAX_SH + 1) / 2; ++q) D[q] = 0.0;
        const double *xb = b < B ? prm[(size_t)s * B + b].xbar : nullptr;
        const double fmean = xb ? xb[0] * 0.28209479177387814 : 0.0;
        if (fmean > 0.0) {
            for (int it = 0; it < rule.nt; ++it) {
                const double z = rule.z[it], rad = sqrt(fmax(0.0, 1.0 - z * z));
                for (int ip = 0; ip < rule.nphi; ++ip) {
                    const double ph = 2.0 * 3.141592653589793 * ip / rule.nphi;
                    float Y[MAXK];
                    sh_eval(order, (float)(rad * cos(ph)), (float)(rad * sin(ph)), (float)z, Y);
                    double f = 0.0;
                    for (int k = 0; k < K; ++k) f += xb[k] * Y[k];
                    const double wa = rule.w[it] * (2.0 * 3.141592653589793 / rule.nphi) * sqrt(fmax(f, 0.0) / fmean);
                    int q = 0;
                    for (int k = 0; k < K; ++k)
                        for (int kp = 0; kp <= k; ++kp) D[q++] += wa * (double)Y[k] * (double)Y[kp];
                }
            }
        }
        int q = 0;
        for (int k = 0; k < RP_MAX_SH; ++k)
            for (int kp = 0; kp < RP_MAX_SH; ++kp) R.D[b][k][kp] = 0.f;
        for (int k = 0; k < K; ++k)
            for (int kp = 0; kp <= k; ++kp, ++q) {
                const float v = (b < B) ? (fmean > 0.0 ? (float)D[q] : (k == kp ? 1.f : 0.f)) : 0.f;
                R.D[b][k][kp] = v;
                R.D[b][kp][k] = v;
            }
    }
    __syncwarp();
    if (lane == 0) {
        R.generation = gen;
        R.mean_delay_s = mu;
        R.resampled = redraw ? 1 : 0;
    }
}

// Gauss-Legendre nodes and weights on [-1, 1] (Newton's method on P_n from the
// three-term recurrence), n <= MAXQ
void gauss_legendre(int n, double *x, double *w)
{
    for (int i = 0; i < n; ++i) {
        double z = std::cos(3.141592653589793 * (i + 0.75) / (n + 0.5));
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            const double pn = n == 1 ? z : p1, pnm1 = n == 1 ? 1.0 : p0;
            const double dp = n * (z * pn - pnm1) / (z * z - 1.0);
            const double dz = pn / dp;
            z -= dz;
            if (std::fabs(dz) < 1e-16) {
                double q0 = 1.0, q1 = z;
                for (int k = 2; k <= n; ++k) {
                    const double q2 = ((2.0 * k - 1.0) * z * q1 - (k - 1.0) * q0) / k;
                    q0 = q1;
                    q1 = q2;
                }
                const double dq = n * (z * q1 - (n == 1 ? 1.0 : q0)) / (z * z - 1.0);
                w[i] = 2.0 / ((1.0 - z * z) * dq * dq);
                break;
            }
        }
        x[i] = z;
    }
}

}  // namespace
}  // namespace rp

extern "C" int rp_reverb_configure(rp_ctx *c, const float *H, const rp_reverb_params *params, int32_t S, int32_t B,
                                   int32_t K, int32_t T, double ir_rate_hz, double mean_free_path,
                                   double speed_of_sound, uint64_t seed, rp_reverberator *rev)
{
    if (!c || !H || !params || !rev || S < 1 || B < 1 || B > RP_MAX_BANDS || T < 1 || !(ir_rate_hz > 0.0) ||
        !(mean_free_path > 0.0) || !(speed_of_sound > 0.0) || !std::isfinite(mean_free_path))
        return RP_ERR_INVALID_ARG;
    const int n = (int)std::lround(std::sqrt((double)K)) - 1;
    if ((n + 1) * (n + 1) != K || n < 0 || n > RP_MAX_SH_ORDER) return RP_ERR_INVALID_ARG;
    if (cudaSetDevice(c->device) != cudaSuccess) return RP_ERR_CUDA;
    SphereRule rule;
    rule.nt = 2 * n + 2;
    rule.nphi = 4 * n + 4;
    gauss_legendre(rule.nt, rule.z, rule.w);
    {
        ProfScope ps(c, "reverb_config");
        k_reverb_config<<<S, 32, 0, c->stream>>>(H, params, S, B, K, T, ir_rate_hz, mean_free_path / speed_of_sound,
                                                  seed, rule, rev);
    }
    return cudaGetLastError() == cudaSuccess ? RP_OK : RP_ERR_CUDA;
}
