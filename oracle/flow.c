/*
 * flow.c -- oracle affine-coupling flow used as a transport map under HMC
 * (the learned preconditioner of this project; the paper's HMC of Sec. 2.1
 * runs in the latent space z with theta = T(z)).  FP64.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * T = layer_{L-1} o ... o layer_0.  Layer l splits z into halves A_l and B_l
 * (even l: A = first half, B = second; odd l: swapped) and maps
 *   b -> b * exp(s(a)) + t(a),   a unchanged,
 * with (s_raw, t) = W3 tanh(W2 tanh(W1 a + b1) + b2) + b3, s = 2 tanh(s_raw).
 * The hidden activation is smooth (tanh, not a ReLU): HMC in the latent space
 * follows grad log pi_z, which contains the derivative of the conditioner,
 * and a ReLU would make that gradient field discontinuous at every kink,
 * breaking the O(eps^2) energy error of Algorithm 1 there.
 * log|det dT/dz| = sum over layers of sum_k s_k.
 * Parameters, per layer, row-major (out x in):
 *   W1 [H x Dh], b1 [H], W2 [H x H], b2 [H], W3 [D x H], b3 [D]   (Dh = D/2;
 *   rows 0..Dh-1 of W3 give s_raw, rows Dh..D-1 give t).
 * Pins (tests/test_oracle_flow.py): T(T^-1(x)) = x; log-determinant against
 * a finite-difference Jacobian determinant; the latent-space gradient and the
 * training-loss gradient against central finite differences; zero last layer
 * gives the identity map.
 */
#include "oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

static int64_t layer_size(int64_t D, int64_t H) {
    const int64_t Dh = D / 2;
    return H * Dh + H + H * H + H + D * H + D;
}

int64_t oracle_flow_num_params(int64_t D, int64_t H, int64_t L) { return L * layer_size(D, H); }

typedef struct {
    const double *W1, *b1, *W2, *b2, *W3, *b3;
} layer_view;

static layer_view view(const oracle_flow* f, int64_t l) {
    const int64_t D = f->D, H = f->H, Dh = D / 2;
    const double* p = f->params + l * layer_size(D, H);
    layer_view v;
    v.W1 = p;
    v.b1 = v.W1 + H * Dh;
    v.W2 = v.b1 + H;
    v.b2 = v.W2 + H * H;
    v.W3 = v.b2 + H;
    v.b3 = v.W3 + D * H;
    return v;
}

/* Indices of the conditioning half A and the transformed half B of layer l. */
static int64_t idx_a(int64_t l, int64_t k, int64_t Dh) { return (l % 2 == 0) ? k : Dh + k; }
static int64_t idx_b(int64_t l, int64_t k, int64_t Dh) { return (l % 2 == 0) ? Dh + k : k; }

/* Conditioner MLP of layer l at the A-half of z: fills h1, h2 (H each) and
 * o (D: s_raw then t). */
static void conditioner(const oracle_flow* f, int64_t l, const double* z, double* h1, double* h2, double* o) {
    const int64_t D = f->D, H = f->H, Dh = D / 2;
    const layer_view v = view(f, l);
    for (int64_t h = 0; h < H; ++h) {
        double acc = v.b1[h];
        for (int64_t k = 0; k < Dh; ++k) acc += v.W1[h * Dh + k] * z[idx_a(l, k, Dh)];
        h1[h] = tanh(acc);
    }
    for (int64_t h = 0; h < H; ++h) {
        double acc = v.b2[h];
        for (int64_t k = 0; k < H; ++k) acc += v.W2[h * H + k] * h1[k];
        h2[h] = tanh(acc);
    }
    for (int64_t r = 0; r < D; ++r) {
        double acc = v.b3[r];
        for (int64_t k = 0; k < H; ++k) acc += v.W3[r * H + k] * h2[k];
        o[r] = acc;
    }
}

void oracle_flow_forward(const oracle_flow* f, const double* z, double* x, double* logdet) {
    const int64_t D = f->D, H = f->H, Dh = D / 2;
    double* h1 = (double*)malloc((size_t)(2 * H + D) * sizeof(double));
    double *h2 = h1 + H, *o = h2 + H;
    memcpy(x, z, (size_t)D * sizeof(double));
    double ld = 0.0;
    for (int64_t l = 0; l < f->L; ++l) {
        conditioner(f, l, x, h1, h2, o);
        for (int64_t k = 0; k < Dh; ++k) {
            const double s = 2.0 * tanh(o[k]), t = o[Dh + k];
            const int64_t ib = idx_b(l, k, Dh);
            x[ib] = x[ib] * exp(s) + t;
            ld += s;
        }
    }
    free(h1);
    if (logdet) *logdet = ld;
}

void oracle_flow_inverse(const oracle_flow* f, const double* x, double* z, double* logdet_inv) {
    const int64_t D = f->D, H = f->H, Dh = D / 2;
    double* h1 = (double*)malloc((size_t)(2 * H + D) * sizeof(double));
    double *h2 = h1 + H, *o = h2 + H;
    memcpy(z, x, (size_t)D * sizeof(double));
    double ld = 0.0;
    for (int64_t l = f->L - 1; l >= 0; --l) {
        conditioner(f, l, z, h1, h2, o);   /* the A-half is the same on both sides */
        for (int64_t k = 0; k < Dh; ++k) {
            const double s = 2.0 * tanh(o[k]), t = o[Dh + k];
            const int64_t ib = idx_b(l, k, Dh);
            z[ib] = (z[ib] - t) * exp(-s);
            ld -= s;
        }
    }
    free(h1);
    if (logdet_inv) *logdet_inv = ld;
}

/* log pi_z(z) = log pi(T(z)) + log|det dT/dz| and its gradient in z:
 * the cotangent grad log pi(x) pulled back through every layer, plus the
 * gradient of the log-determinant. */
double oracle_flow_logpi_z(const oracle_flow* f, const oracle_target* t, const double* z, double* gz,
                           double* x_out, double* gx_out, double* logpi_x_out) {
    const int64_t D = f->D, H = f->H, Dh = D / 2, L = f->L;
    double* zl = (double*)malloc((size_t)(L * D + D + D + 2 * H + D + 3 * H + D) * sizeof(double));
    double* x = zl + L * D;
    double* c = x + D;
    double *h1 = c + D, *h2 = h1 + H, *o = h2 + H;
    double *co = o + D, *ch2 = co + D, *ch1 = ch2 + H, *tmp = ch1 + H;
    (void)tmp;
    memcpy(x, z, (size_t)D * sizeof(double));
    double ld = 0.0;
    for (int64_t l = 0; l < L; ++l) {
        memcpy(zl + l * D, x, (size_t)D * sizeof(double));
        conditioner(f, l, x, h1, h2, o);
        for (int64_t k = 0; k < Dh; ++k) {
            const double s = 2.0 * tanh(o[k]), tt = o[Dh + k];
            const int64_t ib = idx_b(l, k, Dh);
            x[ib] = x[ib] * exp(s) + tt;
            ld += s;
        }
    }
    const double lpx = oracle_logpi(t, x, c);
    if (x_out) memcpy(x_out, x, (size_t)D * sizeof(double));
    if (gx_out) memcpy(gx_out, c, (size_t)D * sizeof(double));
    if (logpi_x_out) *logpi_x_out = lpx;
    if (gz) {
        for (int64_t l = L - 1; l >= 0; --l) {
            const layer_view v = view(f, l);
            const double* in = zl + l * D;
            conditioner(f, l, in, h1, h2, o);
            for (int64_t k = 0; k < Dh; ++k) {
                const int64_t ib = idx_b(l, k, Dh);
                const double th = tanh(o[k]), s = 2.0 * th, es = exp(s);
                const double cbp = c[ib];                         /* cotangent of b' */
                const double cs = cbp * in[ib] * es + 1.0;        /* + d logdet / ds */
                co[k] = cs * 2.0 * (1.0 - th * th);
                co[Dh + k] = cbp;                                 /* d b' / d t = 1 */
                c[ib] = cbp * es;                                 /* cotangent of b */
            }
            for (int64_t h = 0; h < H; ++h) {
                double acc = 0.0;
                for (int64_t r = 0; r < D; ++r) acc += v.W3[r * H + h] * co[r];
                ch2[h] = acc * (1.0 - h2[h] * h2[h]);
            }
            for (int64_t h = 0; h < H; ++h) {
                double acc = 0.0;
                for (int64_t r = 0; r < H; ++r) acc += v.W2[r * H + h] * ch2[r];
                ch1[h] = acc * (1.0 - h1[h] * h1[h]);
            }
            for (int64_t k = 0; k < Dh; ++k) {
                double acc = 0.0;
                for (int64_t h = 0; h < H; ++h) acc += v.W1[h * Dh + k] * ch1[h];
                c[idx_a(l, k, Dh)] += acc;
            }
        }
        memcpy(gz, c, (size_t)D * sizeof(double));
    }
    free(zl);
    return lpx + ld;
}

/* Weighted negative log-likelihood of particles theta (N x D) with
 * normalised weights W under the flow density N(T^-1(theta); 0, I)
 * |det dT^-1/dtheta|, without the constant D/2 log 2 pi:
 *   loss = sum_j W_j (1/2 |z_j|^2 + sum over layers of sum_k s_k),
 * and its gradient with respect to every parameter (back-propagation through
 * the inverse layers). */
double oracle_flow_loss_grad(const oracle_flow* f, const double* theta, const double* W, int64_t N,
                             double* grad) {
    const int64_t D = f->D, H = f->H, Dh = D / 2, L = f->L;
    const int64_t np = oracle_flow_num_params(D, H, L);
    if (grad) memset(grad, 0, (size_t)np * sizeof(double));
    double* ul = (double*)malloc((size_t)(L * D + 2 * D + 3 * H + 2 * D + 2 * H) * sizeof(double));
    double* z = ul + L * D;
    double* c = z + D;
    double *h1 = c + D, *h2 = h1 + H, *o = h2 + H;
    double *co = o + D, *ch2 = co + D, *ch1 = ch2 + H;
    double loss = 0.0;
    for (int64_t j = 0; j < N; ++j) {
        /* a particle of zero weight adds nothing to the weighted loss; its
         * position may be non-finite (the end of a divergent trajectory) */
        if (W[j] == 0.0) continue;
        memcpy(z, theta + j * D, (size_t)D * sizeof(double));
        double ssum = 0.0;
        /* inverse pass, layer L-1 first; ul[l] = input of inverse layer l */
        for (int64_t l = L - 1; l >= 0; --l) {
            memcpy(ul + l * D, z, (size_t)D * sizeof(double));
            conditioner(f, l, z, h1, h2, o);
            for (int64_t k = 0; k < Dh; ++k) {
                const double s = 2.0 * tanh(o[k]), t = o[Dh + k];
                const int64_t ib = idx_b(l, k, Dh);
                z[ib] = (z[ib] - t) * exp(-s);
                ssum += s;
            }
        }
        double zz = 0.0;
        for (int64_t d = 0; d < D; ++d) zz += z[d] * z[d];
        loss += W[j] * (0.5 * zz + ssum);
        if (!grad) continue;
        for (int64_t d = 0; d < D; ++d) c[d] = W[j] * z[d];
        /* back-propagate from layer 0 (the last inverse applied) to L-1 */
        for (int64_t l = 0; l < L; ++l) {
            const layer_view v = view(f, l);
            double* g = grad + l * layer_size(D, H);
            double *gW1 = g, *gb1 = gW1 + H * Dh, *gW2 = gb1 + H, *gb2 = gW2 + H * H, *gW3 = gb2 + H,
                   *gb3 = gW3 + D * H;
            const double* in = ul + l * D;    /* (a, b') */
            conditioner(f, l, in, h1, h2, o);
            for (int64_t k = 0; k < Dh; ++k) {
                const int64_t ib = idx_b(l, k, Dh);
                const double th = tanh(o[k]), s = 2.0 * th, ems = exp(-s);
                const double b = (in[ib] - o[Dh + k]) * ems;  /* output of this inverse layer */
                const double cb = c[ib];
                const double cs = -cb * b + W[j];
                co[k] = cs * 2.0 * (1.0 - th * th);
                co[Dh + k] = -cb * ems;
                c[ib] = cb * ems;                             /* cotangent of b' */
            }
            for (int64_t r = 0; r < D; ++r) {
                gb3[r] += co[r];
                for (int64_t h = 0; h < H; ++h) gW3[r * H + h] += co[r] * h2[h];
            }
            for (int64_t h = 0; h < H; ++h) {
                double acc = 0.0;
                for (int64_t r = 0; r < D; ++r) acc += v.W3[r * H + h] * co[r];
                ch2[h] = acc * (1.0 - h2[h] * h2[h]);
            }
            for (int64_t r = 0; r < H; ++r) {
                gb2[r] += ch2[r];
                for (int64_t h = 0; h < H; ++h) gW2[r * H + h] += ch2[r] * h1[h];
            }
            for (int64_t h = 0; h < H; ++h) {
                double acc = 0.0;
                for (int64_t r = 0; r < H; ++r) acc += v.W2[r * H + h] * ch2[r];
                ch1[h] = acc * (1.0 - h1[h] * h1[h]);
            }
            for (int64_t h = 0; h < H; ++h) {
                gb1[h] += ch1[h];
                for (int64_t k = 0; k < Dh; ++k) gW1[h * Dh + k] += ch1[h] * in[idx_a(l, k, Dh)];
            }
            for (int64_t k = 0; k < Dh; ++k) {
                double acc = 0.0;
                for (int64_t h = 0; h < H; ++h) acc += v.W1[h * Dh + k] * ch1[h];
                c[idx_a(l, k, Dh)] += acc;
            }
        }
    }
    free(ul);
    return loss;
}

void oracle_flow_adam(double* params, const double* grad, double* m, double* v, int64_t n, int32_t t, double lr,
                      double b1, double b2, double eps) {
    /* Adam (Kingma & Ba 2015), descent on the loss; t is the 1-based step. */
    const double c1 = 1.0 - pow(b1, (double)t), c2 = 1.0 - pow(b2, (double)t);
    for (int64_t i = 0; i < n; ++i) {
        m[i] = b1 * m[i] + (1.0 - b1) * grad[i];
        v[i] = b2 * v[i] + (1.0 - b2) * grad[i] * grad[i];
        params[i] -= lr * (m[i] / c1) / (sqrt(v[i] / c2) + eps);
    }
}
