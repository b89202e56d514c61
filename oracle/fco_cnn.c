/*
 * fco_cnn.c -- FP64 forward and backward pass of the learned refinement
 * tagger (TEST INFRASTRUCTURE).  The paper has no learned component; the
 * network stands in for the Sec. 5 tagging criterion and predicts the
 * criterion's flags several steps ahead.
 *
 * Network: input x[3][S][S] (a patch's fields plus both ghost layers),
 *   a1 = relu(conv3x3_valid(x; w1, b1))   16 channels, (S-2)^2
 *   a2 = relu(conv3x3_valid(a1; w2, b2))  16 channels, (S-4)^2
 *   z  = conv3x3_valid(a2; w3, b3)         2 channels, (S-6)^2
 *   logits[c] = max over positions of z[c] (first maximum in raster order).
 * Loss per sample: sum over the two logits of binary cross-entropy with
 * logits; the batch loss is the mean over samples.
 * Convolution: y[o][r][c] = b[o] + sum_i sum_ky sum_kx w[o][i][ky][kx] x[i][r+ky][c+kx].
 */
#include "fco_internal.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

#define C1 16
#define C2 16
#define C3 2

static void conv_fwd(int Ci, int Co, int S, const double *w, const double *b, const double *x, double *y)
{
    int So = S - 2;
    for (int o = 0; o < Co; ++o)
        for (int r = 0; r < So; ++r)
            for (int c = 0; c < So; ++c) {
                double acc = b[o];
                for (int i = 0; i < Ci; ++i)
                    for (int ky = 0; ky < 3; ++ky)
                        for (int kx = 0; kx < 3; ++kx)
                            acc += w[((o * Ci + i) * 3 + ky) * 3 + kx] * x[(i * S + r + ky) * S + c + kx];
                y[(o * So + r) * So + c] = acc;
            }
}

/* given dy, accumulate dw, db and (if dx) write dx */
static void conv_bwd(int Ci, int Co, int S, const double *w, const double *x, const double *dy,
                     double *dw, double *db, double *dx)
{
    int So = S - 2;
    if (dx) memset(dx, 0, sizeof(double) * (size_t)Ci * S * S);
    for (int o = 0; o < Co; ++o)
        for (int r = 0; r < So; ++r)
            for (int c = 0; c < So; ++c) {
                double g = dy[(o * So + r) * So + c];
                if (g == 0.0) continue;
                db[o] += g;
                for (int i = 0; i < Ci; ++i)
                    for (int ky = 0; ky < 3; ++ky)
                        for (int kx = 0; kx < 3; ++kx) {
                            dw[((o * Ci + i) * 3 + ky) * 3 + kx] += g * x[(i * S + r + ky) * S + c + kx];
                            if (dx) dx[(i * S + r + ky) * S + c + kx] += g * w[((o * Ci + i) * 3 + ky) * 3 + kx];
                        }
            }
}

typedef struct { const double *w1, *b1, *w2, *b2, *w3, *b3; } net_t;

static net_t unpack(const double *w)
{
    net_t n;
    n.w1 = w; n.b1 = n.w1 + C1 * 3 * 9;
    n.w2 = n.b1 + C1; n.b2 = n.w2 + C2 * C1 * 9;
    n.w3 = n.b2 + C2; n.b3 = n.w3 + C3 * C2 * 9;
    return n;
}

/* forward of one sample; keeps activations for the backward pass */
static void forward1(const net_t *n, int S, const double *x, double *a1, double *a2, double *z,
                     double *logit, int *arg)
{
    int S1 = S - 2, S2 = S - 4, S3 = S - 6;
    conv_fwd(3, C1, S, n->w1, n->b1, x, a1);
    for (int k = 0; k < C1 * S1 * S1; ++k) a1[k] = a1[k] > 0.0 ? a1[k] : 0.0;
    conv_fwd(C1, C2, S1, n->w2, n->b2, a1, a2);
    for (int k = 0; k < C2 * S2 * S2; ++k) a2[k] = a2[k] > 0.0 ? a2[k] : 0.0;
    conv_fwd(C2, C3, S2, n->w3, n->b3, a2, z);
    for (int c = 0; c < C3; ++c) {
        int best = 0;
        for (int k = 1; k < S3 * S3; ++k)
            if (z[c * S3 * S3 + k] > z[c * S3 * S3 + best]) best = k;
        arg[c] = best;
        logit[c] = z[c * S3 * S3 + best];
    }
}

int fco_cnn_forward(int N, int S, const double *w, const double *x, double *logits)
{
    if (S < 7) return FCO_ERR_ARG;
    net_t n = unpack(w);
    int S1 = S - 2, S2 = S - 4, S3 = S - 6;
    double *a1 = (double *)malloc(sizeof(double) * C1 * S1 * S1);
    double *a2 = (double *)malloc(sizeof(double) * C2 * S2 * S2);
    double *z = (double *)malloc(sizeof(double) * C3 * S3 * S3);
    for (int s = 0; s < N; ++s) {
        int arg[C3];
        forward1(&n, S, x + (size_t)s * 3 * S * S, a1, a2, z, logits + 2 * s, arg);
    }
    free(a1); free(a2); free(z);
    return FCO_OK;
}

/* BCE with logits: softplus(z) - y z, written stably */
static double bce(double z, double y) { return (z > 0.0 ? z : 0.0) - y * z + log1p(exp(-fabs(z))); }
static double sigmoid(double z) { return 1.0 / (1.0 + exp(-z)); }

double fco_cnn_loss_grad(int N, int S, const double *w, const double *x,
                         const double *targets, double *grad)
{
    net_t n = unpack(w);
    int S1 = S - 2, S2 = S - 4, S3 = S - 6;
    double *a1 = (double *)malloc(sizeof(double) * C1 * S1 * S1);
    double *a2 = (double *)malloc(sizeof(double) * C2 * S2 * S2);
    double *z = (double *)malloc(sizeof(double) * C3 * S3 * S3);
    double *dz = (double *)malloc(sizeof(double) * C3 * S3 * S3);
    double *da2 = (double *)malloc(sizeof(double) * C2 * S2 * S2);
    double *da1 = (double *)malloc(sizeof(double) * C1 * S1 * S1);
    memset(grad, 0, sizeof(double) * FCO_CNN_NPARAM);
    double *gw1 = grad, *gb1 = gw1 + C1 * 3 * 9, *gw2 = gb1 + C1, *gb2 = gw2 + C2 * C1 * 9;
    double *gw3 = gb2 + C2, *gb3 = gw3 + C3 * C2 * 9;
    double loss = 0.0;
    for (int s = 0; s < N; ++s) {
        const double *xs = x + (size_t)s * 3 * S * S;
        double logit[C3];
        int arg[C3];
        forward1(&n, S, xs, a1, a2, z, logit, arg);
        memset(dz, 0, sizeof(double) * C3 * S3 * S3);
        for (int c = 0; c < C3; ++c) {
            double y = targets[2 * s + c];
            loss += bce(logit[c], y) / N;
            dz[c * S3 * S3 + arg[c]] = (sigmoid(logit[c]) - y) / N;
        }
        conv_bwd(C2, C3, S2, n.w3, a2, dz, gw3, gb3, da2);
        for (int k = 0; k < C2 * S2 * S2; ++k) if (!(a2[k] > 0.0)) da2[k] = 0.0;
        conv_bwd(C1, C2, S1, n.w2, a1, da2, gw2, gb2, da1);
        for (int k = 0; k < C1 * S1 * S1; ++k) if (!(a1[k] > 0.0)) da1[k] = 0.0;
        conv_bwd(3, C1, S, n.w1, xs, da1, gw1, gb1, NULL);
    }
    free(a1); free(a2); free(z); free(dz); free(da2); free(da1);
    return loss;
}
