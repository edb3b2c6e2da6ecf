/*
 * mlp.c -- FP64 CPU oracle of the learned reverberation-parameter estimator: a
 * multilayer perceptron that maps a low-ray-count energy IR plus scene features to
 * per-band decay times and direct-to-reverberant ratios, its masked mean-squared
 * loss, the gradient of that loss, and the AdamW update.
 *
 * TEST INFRASTRUCTURE ONLY (see oracle.c): used by tests and the benchmark's CPU
 * leg, never by the product path; it shares no code with the CUDA kernels.
 *
 * Network: nh hidden layers of width dh with GELU (exact, x * Phi(x)), linear
 * output of width dout.  Parameters, row-major W[in][out] then b[out], layer after
 * layer:  W1 [din][dh], b1 [dh], W2 [dh][dh], b2 [dh], ..., Wo [dh][dout], bo [dout].
 * Loss: sum over samples and outputs of mask * (y - t)^2, divided by the sum of the
 * mask (at least 1).
 * AdamW: Loshchilov & Hutter (decoupled weight decay), bias-corrected moments.
 * Features: per band the energy-decay curve (the backward energy integral of
 * Section 4.2, "Reverberation Time"), normalised, sampled in a window that ends
 * where it first falls below -40 dB; the window length; the scene features.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static double gelu(double x) { return 0.5 * x * (1.0 + erf(x / sqrt(2.0))); }

static double gelu_grad(double x)
{
    const double phi = exp(-0.5 * x * x) / sqrt(2.0 * 3.14159265358979323846);
    return 0.5 * (1.0 + erf(x / sqrt(2.0))) + x * phi;
}

static int64_t param_count(int din, int dh, int nh, int dout)
{
    int64_t n = (int64_t)din * dh + dh;
    for (int l = 1; l < nh; ++l) n += (int64_t)dh * dh + dh;
    n += (int64_t)dh * dout + dout;
    return n;
}

int64_t orc_mlp_param_count(int din, int dh, int nh, int dout) { return param_count(din, dh, nh, dout); }

/* y[n][out] = x[n][in] W[in][out] + b[out] */
static void affine(int n, int in, int out, const double *x, const double *W, const double *b, double *y)
{
    for (int i = 0; i < n; ++i)
        for (int o = 0; o < out; ++o) {
            double s = b[o];
            for (int k = 0; k < in; ++k) s += x[(int64_t)i * in + k] * W[(int64_t)k * out + o];
            y[(int64_t)i * out + o] = s;
        }
}

/* forward pass keeping every pre-activation z_l and activation a_l (a_0 = x) */
static void forward_all(int n, int din, int dh, int nh, int dout, const double *P, const double *X, double **Z,
                        double **A, double *Y)
{
    const double *p = P;
    const double *in = X;
    int width = din;
    for (int l = 0; l < nh; ++l) {
        affine(n, width, dh, in, p, p + (int64_t)width * dh, Z[l]);
        for (int64_t i = 0; i < (int64_t)n * dh; ++i) A[l][i] = gelu(Z[l][i]);
        p += (int64_t)width * dh + dh;
        in = A[l];
        width = dh;
    }
    affine(n, width, dout, in, p, p + (int64_t)width * dout, Y);
}

void orc_mlp_forward(int n, int din, int dh, int nh, int dout, const double *P, const double *X, double *Y)
{
    double **Z = (double **)malloc(sizeof(double *) * nh), **A = (double **)malloc(sizeof(double *) * nh);
    for (int l = 0; l < nh; ++l) {
        Z[l] = (double *)malloc(sizeof(double) * (size_t)n * dh);
        A[l] = (double *)malloc(sizeof(double) * (size_t)n * dh);
    }
    forward_all(n, din, dh, nh, dout, P, X, Z, A, Y);
    for (int l = 0; l < nh; ++l) {
        free(Z[l]);
        free(A[l]);
    }
    free(Z);
    free(A);
}

/* masked MSE loss and its gradient with respect to every parameter (same layout) */
double orc_mlp_loss_grad(int n, int din, int dh, int nh, int dout, const double *P, const double *X,
                         const double *Tg, const double *mask, double *G)
{
    double **Z = (double **)malloc(sizeof(double *) * nh), **A = (double **)malloc(sizeof(double *) * nh);
    for (int l = 0; l < nh; ++l) {
        Z[l] = (double *)malloc(sizeof(double) * (size_t)n * dh);
        A[l] = (double *)malloc(sizeof(double) * (size_t)n * dh);
    }
    double *Y = (double *)malloc(sizeof(double) * (size_t)n * dout);
    forward_all(n, din, dh, nh, dout, P, X, Z, A, Y);
    double msum = 0.0, loss = 0.0;
    for (int64_t i = 0; i < (int64_t)n * dout; ++i) msum += mask[i];
    const double norm = msum > 1.0 ? msum : 1.0;
    /* dL/dy */
    double *dY = (double *)malloc(sizeof(double) * (size_t)n * dout);
    for (int64_t i = 0; i < (int64_t)n * dout; ++i) {
        const double r = Y[i] - Tg[i];
        loss += mask[i] * r * r;
        dY[i] = 2.0 * mask[i] * r / norm;
    }
    loss /= norm;
    memset(G, 0, sizeof(double) * (size_t)param_count(din, dh, nh, dout));
    /* parameter offsets of each layer */
    int64_t *off = (int64_t *)malloc(sizeof(int64_t) * (nh + 1));
    int64_t o = 0;
    for (int l = 0; l <= nh; ++l) {
        const int in = l == 0 ? din : dh, out = l == nh ? dout : dh;
        off[l] = o;
        o += (int64_t)in * out + out;
    }
    /* backward through the output layer and the hidden layers */
    double *delta = dY; /* dL/d(pre-activation) of the current layer */
    int out = dout;
    for (int l = nh; l >= 0; --l) {
        const int in = l == 0 ? din : dh;
        const double *a_in = l == 0 ? X : A[l - 1];
        double *gW = G + off[l], *gb = G + off[l] + (int64_t)in * out;
        for (int i = 0; i < n; ++i)
            for (int c = 0; c < out; ++c) {
                const double dv = delta[(int64_t)i * out + c];
                gb[c] += dv;
                for (int k = 0; k < in; ++k) gW[(int64_t)k * out + c] += a_in[(int64_t)i * in + k] * dv;
            }
        if (l == 0) break;
        /* delta of the previous layer: (delta W^T) * gelu'(z) */
        const double *W = P + off[l];
        double *prev = (double *)malloc(sizeof(double) * (size_t)n * in);
        for (int i = 0; i < n; ++i)
            for (int k = 0; k < in; ++k) {
                double s = 0.0;
                for (int c = 0; c < out; ++c) s += delta[(int64_t)i * out + c] * W[(int64_t)k * out + c];
                prev[(int64_t)i * in + k] = s * gelu_grad(Z[l - 1][(int64_t)i * in + k]);
            }
        if (delta != dY) free(delta);
        delta = prev;
        out = in;
    }
    if (delta != dY) free(delta);
    free(dY);
    free(off);
    for (int l = 0; l < nh; ++l) {
        free(Z[l]);
        free(A[l]);
    }
    free(Z);
    free(A);
    free(Y);
    return loss;
}

/* one AdamW step over `count` parameters (step counts from 1) */
void orc_adamw_step(int64_t count, double *p, const double *g, double *m, double *v, double lr, double beta1,
                    double beta2, double eps, double wd, int step)
{
    const double c1 = 1.0 - pow(beta1, step), c2 = 1.0 - pow(beta2, step);
    for (int64_t i = 0; i < count; ++i) {
        m[i] = beta1 * m[i] + (1.0 - beta1) * g[i];
        v[i] = beta2 * v[i] + (1.0 - beta2) * g[i] * g[i];
        const double mh = m[i] / c1, vh = v[i] / c2;
        p[i] -= lr * (mh / (sqrt(vh) + eps) + wd * p[i]);
    }
}

/* Input features of S samples of H[S][B][K][T] (only the k = 0 series is read).
 * Per band b < 8: D(t) = sum_{t' >= t} h(t'), r(t) = D(t) / D(0) (0 when D(0) = 0);
 * t_end = first t with r(t) < 1e-4 (T if none), at least 4; for i = 0..62 the
 * position p = t_end (i + 1) / 63, clamped to T - 1.001, and
 * X[b*64 + i] = log10(r(floor p) (1 - w) + r(min(floor p + 1, T - 1)) w + 1e-8) with
 * w = p - floor p; X[b*64 + 63] = ln(t_end / ir_rate).  Bands b >= B are empty bands.
 * scene[S][10] goes to X[512..521], zeros to the end of the row (in_dim). */
void orc_mlp_features(int S, int B, int K, int T, double ir_rate, const double *H, const double *scene, int in_dim,
                      double *X)
{
    double *r = (double *)malloc(sizeof(double) * (size_t)T);
    for (int s = 0; s < S; ++s) {
        double *x = X + (int64_t)s * in_dim;
        for (int b = 0; b < 8; ++b) {
            double D = 0.0;
            for (int t = T - 1; t >= 0; --t) {
                if (b < B) D += H[(((int64_t)s * B + b) * K + 0) * T + t];
                r[t] = D;
            }
            const double D0 = r[0];
            for (int t = 0; t < T; ++t) r[t] = D0 > 0.0 ? r[t] / D0 : 0.0;
            int first = T;
            for (int t = 0; t < T; ++t)
                if (r[t] < 1e-4) {
                    first = t;
                    break;
                }
            const double t_end = first < 4 ? 4.0 : (double)first;
            for (int i = 0; i < 63; ++i) {
                double p = t_end * (i + 1) / 63.0;
                if (p > T - 1.001) p = T - 1.001;
                const int i0 = (int)floor(p);
                const int i1 = i0 + 1 < T ? i0 + 1 : T - 1;
                const double w = p - i0;
                x[b * 64 + i] = log10(r[i0] * (1.0 - w) + r[i1] * w + 1e-8);
            }
            x[b * 64 + 63] = log(t_end / ir_rate);
        }
        for (int f = 0; f < 10; ++f) x[512 + f] = scene[(int64_t)s * 10 + f];
        for (int f = 522; f < in_dim; ++f) x[f] = 0.0;
    }
    free(r);
}
