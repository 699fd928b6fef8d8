/*
 * qqa_oracle.c -- plain FP64 CPU oracle for Parallel Quasi-Quantum Annealing
 * (Ichikawa & Arai, "Optimization by Parallel Quasi-Quantum Annealing with
 * Gradient-Based Sampling", arXiv 2409.02135).
 *
 * TEST INFRASTRUCTURE. This file is the reference the CUDA path is checked
 * against. Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline /
 * reference legs may load it. It shares no code, header or table with the
 * CUDA library, and the CUDA library never calls it.
 *
 * Everything is FP64 and written as the paper states it, one (node, replica)
 * element at a time, with no blocking or fusion:
 *   - energies l(x) and their relaxations l^(p)   (Eq. 2; Sec. 3.1; App. D.1 Eqs. 22, 24, 26)
 *   - alpha-entropy s(p) and the gamma schedule   (Eq. 7; Sec. 5 "Implementation"; App. C.2)
 *   - communication term -S*alpha*sum_i STD_i     (Eq. 10, Sec. 3.3)
 *   - sensitive transition + AdamW + Langevin noise + clamp (Eq. 11, Sec. 3.4, Sec. 5, App. C.3)
 *   - projection rounding x = Theta(p - 1/2) and exact integer costs (Sec. 5 "Implementation")
 *
 * Layout: X[i*S + s] = p_i^{(s)} (node-major, S contiguous), CSR adjacency
 * (row_ptr[n+1], col[nnz], optional integer weights w[nnz]; NULL = unit).
 *
 * Readings where the paper is silent:
 *   - STD uses the population normalisation of Eq. 10 and sqrt(var + comm_eps)
 *     so the derivative exists when all S values coincide.
 *   - AdamW: decoupled weight decay p *= 1 - lr*wd, then the bias-corrected
 *     Adam step with step count t+1 (beta1, beta2, eps are parameters).
 *   - Noise sqrt(2*lr*T)*xi is added after the optimizer step, before the clamp.
 *   - gamma_t = gamma_min + (gamma_max - gamma_min) * t/(K-1), t = 0..K-1.
 *   - Initial p ~ U(0,1] drawn from the counter RNG below.
 *   - Rounding x_i = 1 iff p_i > 1/2 (strict).
 *   - Random numbers: Philox4x32-10 (Salmon et al., SC'11). key = seed,
 *     counter = (node i, replica quad s/4, step t, tag) with tag 0 = init,
 *     1 = noise. u = ((r >> 8) + 1) * 2^-24 in (0,1]; Gaussians by
 *     Box-Muller on consecutive uniform pairs.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MIS 0
#define OR_MAXCUT 1
#define OR_MAXCLIQUE 2

typedef struct {
    int32_t kind;       /* OR_MIS / OR_MAXCUT / OR_MAXCLIQUE */
    int32_t S;          /* replicas */
    int32_t K;          /* annealing steps */
    int32_t a_ent;      /* alpha-entropy exponent (even) */
    double lr, weight_decay, beta1, beta2, adam_eps;
    double gamma_min, gamma_max;
    double alpha_comm, comm_eps;
    double temperature;
    double lambda;      /* penalty coefficient */
    uint64_t seed;
} oracle_params;

/* ------------------------------------------------------------------ */
/* Philox4x32-10, written from Salmon, Moraes, Dror & Shaw (SC'11).   */
/* ------------------------------------------------------------------ */
void oracle_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4])
{
    uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
    uint32_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        uint64_t prod0 = (uint64_t)0xD2511F53u * (uint64_t)c0;
        uint64_t prod1 = (uint64_t)0xCD9E8D57u * (uint64_t)c2;
        uint32_t hi0 = (uint32_t)(prod0 >> 32), lo0 = (uint32_t)prod0;
        uint32_t hi1 = (uint32_t)(prod1 >> 32), lo1 = (uint32_t)prod1;
        uint32_t n0 = hi1 ^ c1 ^ k0;
        uint32_t n1 = lo1;
        uint32_t n2 = hi0 ^ c3 ^ k1;
        uint32_t n3 = lo0;
        c0 = n0; c1 = n1; c2 = n2; c3 = n3;
        k0 += 0x9E3779B9u;   /* Weyl key schedule */
        k1 += 0xBB67AE85u;
    }
    out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

static double u01_from_bits(uint32_t r)
{
    return ((double)((r >> 8) + 1u)) * (1.0 / 16777216.0);
}

static void draw4(uint64_t seed, uint32_t i, uint32_t quad, uint32_t t, uint32_t tag, uint32_t out[4])
{
    uint32_t ctr[4] = {i, quad, t, tag};
    uint32_t key[2] = {(uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32)};
    oracle_philox4x32_10(ctr, key, out);
}

/* uniform in (0,1] used for the initial state, element (i, s) */
double oracle_uniform(uint64_t seed, int32_t i, int32_t s, int32_t t, int32_t tag)
{
    uint32_t r[4];
    draw4(seed, (uint32_t)i, (uint32_t)(s / 4), (uint32_t)t, (uint32_t)tag, r);
    return u01_from_bits(r[s % 4]);
}

/* standard normal xi for element (i, s) at step t (Box-Muller) */
double oracle_gaussian(uint64_t seed, int32_t i, int32_t s, int32_t t)
{
    uint32_t r[4];
    draw4(seed, (uint32_t)i, (uint32_t)(s / 4), (uint32_t)t, 1u, r);
    int pair = (s % 4) / 2;          /* (r0,r1) feed s%4 in {0,1}; (r2,r3) feed {2,3} */
    double u1 = u01_from_bits(r[2 * pair]);
    double u2 = u01_from_bits(r[2 * pair + 1]);
    double radius = sqrt(-2.0 * log(u1));
    double angle = 2.0 * M_PI * u2;
    return (s % 2 == 0) ? radius * cos(angle) : radius * sin(angle);
}

/* xi[i*S + s] = standard normal of element (i, s) at step t, for all elements */
void oracle_noise_field(int32_t n, int32_t S, uint64_t seed, int32_t t, double *xi)
{
    for (int32_t i = 0; i < n; ++i)
        for (int32_t s = 0; s < S; ++s) xi[(int64_t)i * S + s] = oracle_gaussian(seed, i, s, t);
}

/* ------------------------------------------------------------------ */
/* Schedule and entropy (Eq. 7, Sec. 5, App. C.2)                      */
/* ------------------------------------------------------------------ */
double oracle_gamma(const oracle_params *P, int32_t t)
{
    if (P->K <= 1) return P->gamma_min;
    return P->gamma_min + (P->gamma_max - P->gamma_min) * (double)t / (double)(P->K - 1);
}

static double ipow(double x, int e)
{
    double r = 1.0;
    for (int k = 0; k < e; ++k) r *= x;
    return r;
}

/* s(p) = sum_i 1 - (2 p_i - 1)^a for one replica vector p[0..n) with stride */
static double entropy_column(int32_t n, const double *X, int32_t S, int32_t s, int a)
{
    double acc = 0.0;
    for (int32_t i = 0; i < n; ++i) acc += 1.0 - ipow(2.0 * X[(int64_t)i * S + s] - 1.0, a);
    return acc;
}

double oracle_entropy(int32_t n, const double *p, int32_t a_ent)
{
    return entropy_column(n, p, 1, 0, a_ent);
}

/* ------------------------------------------------------------------ */
/* Energies (App. D.1) and their relaxations (Sec. 3.1)                */
/* ------------------------------------------------------------------ */
static double edge_w(const int32_t *w, int64_t k) { return w ? (double)w[k] : 1.0; }

/* relaxed loss l^(p) for one replica column (p may be binary: l^(x) = l(x)) */
static double relaxed_loss_column(int32_t kind, int32_t n, const int32_t *rp, const int32_t *col,
                                  const int32_t *w, double lambda, const double *X, int32_t S, int32_t s)
{
    double sum_p = 0.0, quad = 0.0;  /* quad = p^T A p = 2 * sum over undirected edges */
    for (int32_t i = 0; i < n; ++i) {
        double pi = X[(int64_t)i * S + s];
        sum_p += pi;
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k)
            quad += edge_w(w, k) * pi * X[(int64_t)col[k] * S + s];
    }
    if (kind == OR_MIS) {
        /* l = -c^T x + lambda * x^T A x / 2, c = 1 */
        return -sum_p + lambda * quad / 2.0;
    } else if (kind == OR_MAXCLIQUE) {
        /* l = -c^T x + lambda/2 * (1^T x (1^T x - 1) - x^T A x) */
        return -sum_p + lambda / 2.0 * (sum_p * (sum_p - 1.0) - quad);
    } else {
        /* l = - sum_{(i,j) in E} A_ij (1 - (2x_i-1)(2x_j-1)) / 2, each edge once */
        double acc = 0.0;
        for (int32_t i = 0; i < n; ++i)
            for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
                int32_t j = col[k];
                if (j <= i) continue;
                double zi = 2.0 * X[(int64_t)i * S + s] - 1.0;
                double zj = 2.0 * X[(int64_t)j * S + s] - 1.0;
                acc += edge_w(w, k) * (1.0 - zi * zj) / 2.0;
            }
        return -acc;
    }
}

double oracle_relaxed_loss(int32_t kind, int32_t n, const int32_t *rp, const int32_t *col,
                           const int32_t *w, double lambda, const double *p)
{
    return relaxed_loss_column(kind, n, rp, col, w, lambda, p, 1, 0);
}

/* population STD of row i over the S replicas, regularised by comm_eps (Eq. 10) */
static void row_stats(const double *X, int32_t S, int32_t i, double comm_eps, double *mean, double *std)
{
    double acc = 0.0;
    for (int32_t s = 0; s < S; ++s) acc += X[(int64_t)i * S + s];
    double m = acc / (double)S;
    double var = 0.0;
    for (int32_t s = 0; s < S; ++s) {
        double d = X[(int64_t)i * S + s] - m;
        var += d * d;
    }
    var /= (double)S;
    *mean = m;
    *std = sqrt(var + comm_eps);
}

/*
 * R({p^(s)}) = sum_s [ l^(p^(s)) + gamma s(p^(s)) ] - S alpha sum_i STD_i    (Eq. 6 and Eq. 10)
 */
double oracle_objective(const oracle_params *P, int32_t n, const int32_t *rp, const int32_t *col,
                        const int32_t *w, double gamma, const double *X)
{
    int32_t S = P->S;
    double total = 0.0;
    for (int32_t s = 0; s < S; ++s) {
        total += relaxed_loss_column(P->kind, n, rp, col, w, P->lambda, X, S, s);
        total += gamma * entropy_column(n, X, S, s, P->a_ent);
    }
    double comm = 0.0;
    for (int32_t i = 0; i < n; ++i) {
        double m, sd;
        row_stats(X, S, i, P->comm_eps, &m, &sd);
        comm += sd;
    }
    return total - (double)S * P->alpha_comm * comm;
}

/*
 * Gradient of R with respect to p_i^{(s)} (derived from the energies of App. D.1):
 *   MIS    : -1 + lambda (A p)_i
 *   clique : -1 + lambda (sum_k p_k - 1/2 - (A p)_i)
 *   cut    : sum_j A_ij (2 p_j - 1) = 2 (A p)_i - d_i
 *   entropy: gamma * (-2 a (2 p_i - 1)^(a-1))
 *   comm   : -alpha (p_i - mean_i) / STD_i   (the S prefactor cancels the 1/S of STD)
 * If gabs != NULL it receives the sum of absolute values of the terms that
 * enter each element (a scale for rounding-error tolerances in tests).
 */
void oracle_gradient_rows(const oracle_params *P, int32_t n, const int32_t *rp, const int32_t *col,
                          const int32_t *w, double gamma, const double *X,
                          const int32_t *rows, int32_t nrows, double *G, double *gabs)
{
    int32_t S = P->S;
    double *colsum = NULL;
    if (P->kind == OR_MAXCLIQUE) {
        colsum = (double *)calloc((size_t)S, sizeof(double));
        for (int32_t i = 0; i < n; ++i)
            for (int32_t s = 0; s < S; ++s) colsum[s] += X[(int64_t)i * S + s];
    }
    #pragma omp parallel for schedule(static)
    for (int32_t r = 0; r < nrows; ++r) {
        int32_t i = rows ? rows[r] : r;
        double mean = 0.0, sd = 1.0;
        if (P->alpha_comm != 0.0) row_stats(X, S, i, P->comm_eps, &mean, &sd);
        for (int32_t s = 0; s < S; ++s) {
            double p = X[(int64_t)i * S + s];
            double Y = 0.0, Yabs = 0.0, deg = 0.0;
            for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
                double term = edge_w(w, k) * X[(int64_t)col[k] * S + s];
                Y += term;
                Yabs += fabs(term);
                deg += edge_w(w, k);
            }
            double g, scale;
            if (P->kind == OR_MIS) {
                g = -1.0 + P->lambda * Y;
                scale = 1.0 + P->lambda * Yabs;
            } else if (P->kind == OR_MAXCLIQUE) {
                g = -1.0 + P->lambda * (colsum[s] - 0.5 - Y);
                scale = 1.0 + P->lambda * (fabs(colsum[s]) + 0.5 + Yabs);
            } else {
                g = 2.0 * Y - deg;
                scale = 2.0 * Yabs + fabs(deg);
            }
            double u = 2.0 * p - 1.0;
            double ent = gamma * (-2.0 * (double)P->a_ent * ipow(u, P->a_ent - 1));
            g += ent;
            scale += fabs(ent);
            if (P->alpha_comm != 0.0) {
                double c = -P->alpha_comm * (p - mean) / sd;
                g += c;
                scale += P->alpha_comm * (fabs(p) + fabs(mean)) / sd;
            }
            G[(int64_t)r * S + s] = g;
            if (gabs) gabs[(int64_t)r * S + s] = scale;
        }
    }
    free(colsum);
}

void oracle_gradient(const oracle_params *P, int32_t n, const int32_t *rp, const int32_t *col,
                     const int32_t *w, double gamma, const double *X, double *G)
{
    oracle_gradient_rows(P, n, rp, col, w, gamma, X, NULL, n, G, NULL);
}

/*
 * One annealing step t for the listed rows (all rows if rows == NULL), Jacobi
 * style: every gradient is taken at the state X = p^t.
 *   Xn_rows, m_rows, v_rows are [nrows][S]; m_rows/v_rows hold the moments of
 *   those rows on entry and are overwritten with the new moments.
 *   grad_rows / gabs_rows (optional) receive g and its term scale.
 * Steps (Eq. 11 with AdamW replacing -eta*grad, Sec. 3.4; clamp Sec. 5; T, wd App. C.3):
 *   p' = p (1 - lr wd)                                 decoupled weight decay
 *   m  = b1 m + (1 - b1) g ;  v = b2 v + (1 - b2) g^2
 *   p' = p' - (lr / bc1) m / (sqrt(v) / sqrt(bc2) + eps),  bc_k = 1 - b_k^(t+1)
 *   p' = p' + sqrt(2 lr T) xi                          Langevin noise
 *   p^{t+1} = clamp(p', 0, 1)
 */
void oracle_step_rows(const oracle_params *P, int32_t n, const int32_t *rp, const int32_t *col,
                      const int32_t *w, int32_t t, const double *X, const int32_t *rows, int32_t nrows,
                      double *Xn_rows, double *m_rows, double *v_rows, double *grad_rows, double *gabs_rows)
{
    int32_t S = P->S;
    double gamma = oracle_gamma(P, t);
    double *G = (double *)malloc(sizeof(double) * (size_t)nrows * (size_t)S);
    double *Gs = (double *)malloc(sizeof(double) * (size_t)nrows * (size_t)S);
    oracle_gradient_rows(P, n, rp, col, w, gamma, X, rows, nrows, G, Gs);
    double bc1 = 1.0 - pow(P->beta1, (double)(t + 1));
    double bc2 = 1.0 - pow(P->beta2, (double)(t + 1));
    double noise_scale = sqrt(2.0 * P->lr * P->temperature);
    #pragma omp parallel for schedule(static)
    for (int32_t r = 0; r < nrows; ++r) {
        int32_t i = rows ? rows[r] : r;
        for (int32_t s = 0; s < S; ++s) {
            int64_t e = (int64_t)r * S + s;
            double g = G[e];
            double p = X[(int64_t)i * S + s];
            double pn = p * (1.0 - P->lr * P->weight_decay);
            double m = P->beta1 * m_rows[e] + (1.0 - P->beta1) * g;
            double v = P->beta2 * v_rows[e] + (1.0 - P->beta2) * g * g;
            double denom = sqrt(v) / sqrt(bc2) + P->adam_eps;
            pn -= (P->lr / bc1) * m / denom;
            if (noise_scale != 0.0) pn += noise_scale * oracle_gaussian(P->seed, i, s, t);
            if (pn < 0.0) pn = 0.0;
            if (pn > 1.0) pn = 1.0;
            Xn_rows[e] = pn;
            m_rows[e] = m;
            v_rows[e] = v;
            if (grad_rows) grad_rows[e] = g;
            if (gabs_rows) gabs_rows[e] = Gs[e];
        }
    }
    free(G);
    free(Gs);
}

/* initial state: p_i^{(s)} ~ U(0,1] from the counter RNG (tag 0), m = v = 0 */
void oracle_init(int32_t n, int32_t S, uint64_t seed, double *X)
{
    for (int32_t i = 0; i < n; ++i)
        for (int32_t s = 0; s < S; ++s) X[(int64_t)i * S + s] = oracle_uniform(seed, i, s, 0, 0);
}

/* ------------------------------------------------------------------ */
/* Exact integer costs of binary vectors (App. D.1)                    */
/* ------------------------------------------------------------------ */
/*
 * Cost of one binary vector x[0..n) (bytes 0/1).
 *   obj:  MIS / clique -> |x| ; cut -> cut weight
 *   viol: MIS -> edges inside x ; clique -> missing edges inside x ; cut -> 0
 *   returns feasible (viol == 0); *energy = l(x) with penalty lambda.
 */
int oracle_cost_of_x(int32_t kind, int32_t n, const int32_t *rp, const int32_t *col, const int32_t *w,
                     double lambda, const uint8_t *x, int64_t *obj, int64_t *viol, double *energy)
{
    int64_t size = 0, inside = 0, cut = 0;
    for (int32_t i = 0; i < n; ++i) {
        size += x[i];
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
            int32_t j = col[k];
            if (j <= i) continue;                       /* each undirected edge once */
            int64_t wk = w ? (int64_t)w[k] : 1;
            if (x[i] && x[j]) inside += 1;
            if (x[i] != x[j]) cut += wk;
        }
    }
    if (kind == OR_MIS) {
        *obj = size; *viol = inside;
        *energy = -(double)size + lambda * (double)inside;
    } else if (kind == OR_MAXCLIQUE) {
        int64_t missing = size * (size - 1) / 2 - inside;
        *obj = size; *viol = missing;
        *energy = -(double)size + lambda * (double)missing;
    } else {
        *obj = cut; *viol = 0;
        *energy = -(double)cut;
    }
    return *viol == 0;
}

/* projection rounding x = Theta(p - 1/2) (strict) of every replica and its costs;
 * best = feasible replica with the largest objective, ties -> lowest s; -1 if none */
int32_t oracle_round_eval(int32_t kind, int32_t n, const int32_t *rp, const int32_t *col, const int32_t *w,
                          double lambda, int32_t S, const double *X,
                          int64_t *obj, int64_t *viol, uint8_t *feasible, double *energy)
{
    uint8_t *x = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
    int32_t best = -1;
    for (int32_t s = 0; s < S; ++s) {
        for (int32_t i = 0; i < n; ++i) x[i] = X[(int64_t)i * S + s] > 0.5 ? 1 : 0;
        feasible[s] = (uint8_t)oracle_cost_of_x(kind, n, rp, col, w, lambda, x, &obj[s], &viol[s], &energy[s]);
        if (feasible[s] && (best < 0 || obj[s] > obj[best])) best = s;
    }
    free(x);
    return best;
}

/*
 * Full run: init, K steps, periodic evaluation every round_every steps (if > 0)
 * and a final evaluation. hist_best[e] receives the best feasible objective
 * after evaluation e (INT64_MIN if no replica is feasible); returns the number
 * of evaluations written (capacity hist_cap). Final per-replica results go to
 * obj/viol/feasible/energy; the final state to X_out (optional).
 */
int32_t oracle_anneal(const oracle_params *P, int32_t n, const int32_t *rp, const int32_t *col,
                      const int32_t *w, int32_t round_every, int32_t steps_to_run,
                      int64_t *obj, int64_t *viol, uint8_t *feasible, double *energy, int32_t *best_out,
                      int64_t *hist_best, int32_t hist_cap, double *X_out)
{
    int32_t S = P->S;
    size_t NS = (size_t)n * (size_t)S;
    double *Xa = (double *)malloc(sizeof(double) * (NS ? NS : 1));
    double *Xb = (double *)malloc(sizeof(double) * (NS ? NS : 1));
    double *m = (double *)calloc(NS ? NS : 1, sizeof(double));
    double *v = (double *)calloc(NS ? NS : 1, sizeof(double));
    oracle_init(n, S, P->seed, Xa);
    int32_t steps = steps_to_run >= 0 ? steps_to_run : P->K;
    int32_t nh = 0;
    for (int32_t t = 0; t < steps; ++t) {
        oracle_step_rows(P, n, rp, col, w, t, Xa, NULL, n, Xb, m, v, NULL, NULL);
        double *tmp = Xa; Xa = Xb; Xb = tmp;
        if (round_every > 0 && (t + 1) % round_every == 0 && t + 1 < steps && nh < hist_cap) {
            int32_t b = oracle_round_eval(P->kind, n, rp, col, w, P->lambda, S, Xa, obj, viol, feasible, energy);
            hist_best[nh++] = b >= 0 ? obj[b] : INT64_MIN;
        }
    }
    int32_t b = oracle_round_eval(P->kind, n, rp, col, w, P->lambda, S, Xa, obj, viol, feasible, energy);
    if (hist_cap > nh && hist_best) hist_best[nh++] = b >= 0 ? obj[b] : INT64_MIN;
    *best_out = b;
    if (X_out) memcpy(X_out, Xa, sizeof(double) * NS);
    free(Xa); free(Xb); free(m); free(v);
    return nh;
}

/* ================================================================== */
/* Categorical PQQA for graph colouring (App. B; Clamp-normalise of     */
/* App. C.4; the colouring energy of App. D.1 with the sign that       */
/* minimises conflicts).                                                */
/*                                                                      */
/* State W[i][k][s] in [0,1] (node i, colour k, replica s), flattened   */
/* as ((i * K + k) * S + s). sigma_ik = W_ik / sum_k' W_ik' (the clamp  */
/* is the identity on [0,1]; a row of zeros maps to 1/K).               */
/* Readings where the paper is silent:                                   */
/*   - after each update W is projected to [0,1], as p is in the binary */
/*     method; sigma is re-formed from the projected W;                 */
/*   - the communication term acts on sigma, per (node, colour), over   */
/*     the S replicas;                                                  */
/*   - random numbers use the binary counters with row index i*K + k;   */
/*   - rounding: x_i = argmax_k sigma_ik, ties to the lowest colour.    */
/* ================================================================== */

/* c_K of the categorical alpha-entropy (App. B): 1 / ((K-1)((K-1)^(a-1) + 1)) */
static double color_cK(int32_t K, int32_t a)
{
    return 1.0 / ((double)(K - 1) * (ipow((double)(K - 1), a - 1) + 1.0));
}

/* sigma of row (i, s): out[k] for k < K; returns the row sum of W (0: uniform) */
static double color_sigma_row(const double *W, int32_t K, int32_t S, int32_t i, int32_t s, double *out)
{
    double sum = 0.0;
    for (int32_t k = 0; k < K; ++k) sum += W[((int64_t)i * K + k) * S + s];
    for (int32_t k = 0; k < K; ++k) out[k] = sum > 0.0 ? W[((int64_t)i * K + k) * S + s] / sum : 1.0 / (double)K;
    return sum;
}

/* s_K(sigma) = sum_i { 1 - c_K sum_k (K sigma_ik - 1)^a }, sigma[n][K] */
double oracle_color_entropy(int32_t n, int32_t K, const double *sig, int32_t a)
{
    double cK = color_cK(K, a), acc = 0.0;
    for (int32_t i = 0; i < n; ++i) {
        double inner = 0.0;
        for (int32_t k = 0; k < K; ++k) inner += ipow((double)K * sig[(int64_t)i * K + k] - 1.0, a);
        acc += 1.0 - cK * inner;
    }
    return acc;
}

/* relaxed conflicts: sum over edges {i, j} (each once) of sum_k sigma_ik sigma_jk, sigma[n][K] */
double oracle_color_relaxed_conflicts(int32_t n, int32_t K, const int32_t *rp, const int32_t *col, const double *sig)
{
    double acc = 0.0;
    for (int32_t i = 0; i < n; ++i)
        for (int32_t e = rp[i]; e < rp[i + 1]; ++e) {
            int32_t j = col[e];
            if (j <= i) continue;
            for (int32_t k = 0; k < K; ++k) acc += sig[(int64_t)i * K + k] * sig[(int64_t)j * K + k];
        }
    return acc;
}

/* conflicts of a colouring x[n]: edges {i, j} with x_i = x_j */
int64_t oracle_color_conflicts(int32_t n, const int32_t *rp, const int32_t *col, const int32_t *x)
{
    int64_t c = 0;
    for (int32_t i = 0; i < n; ++i)
        for (int32_t e = rp[i]; e < rp[i + 1]; ++e)
            if (col[e] > i && x[col[e]] == x[i]) ++c;
    return c;
}

/* population mean and STD_eps of sigma_ik over the replicas (Eq. 10) */
static void color_stats(const double *SIG, int32_t K, int32_t S, int32_t i, int32_t k, double comm_eps, double *mean,
                        double *std)
{
    double acc = 0.0;
    for (int32_t s = 0; s < S; ++s) acc += SIG[((int64_t)i * K + k) * S + s];
    double m = acc / (double)S, var = 0.0;
    for (int32_t s = 0; s < S; ++s) {
        double d = SIG[((int64_t)i * K + k) * S + s] - m;
        var += d * d;
    }
    *mean = m;
    *std = sqrt(var / (double)S + comm_eps);
}

/* sigma of every (i, k, s) from W, same layout */
static void color_sigma_all(int32_t n, int32_t K, int32_t S, const double *W, double *SIG)
{
    double *row = (double *)malloc(sizeof(double) * (size_t)K);
    for (int32_t i = 0; i < n; ++i)
        for (int32_t s = 0; s < S; ++s) {
            color_sigma_row(W, K, S, i, s, row);
            for (int32_t k = 0; k < K; ++k) SIG[((int64_t)i * K + k) * S + s] = row[k];
        }
    free(row);
}

/*
 * R(W) = sum_s [ conflicts^(sigma_s) + gamma s_K(sigma_s) ] - S alpha sum_{i,k} STD_ik,
 * sigma = Clamp-normalise(W) (App. B, App. C.4, Eq. 10).
 */
double oracle_color_objective(const oracle_params *P, int32_t n, int32_t K, const int32_t *rp, const int32_t *col,
                              double gamma, const double *W)
{
    int32_t S = P->S;
    size_t NKS = (size_t)n * (size_t)K * (size_t)S;
    double *SIG = (double *)malloc(sizeof(double) * (NKS ? NKS : 1));
    double *col_sig = (double *)malloc(sizeof(double) * ((size_t)n * K ? (size_t)n * K : 1));
    color_sigma_all(n, K, S, W, SIG);
    double total = 0.0;
    for (int32_t s = 0; s < S; ++s) {
        for (int32_t i = 0; i < n; ++i)
            for (int32_t k = 0; k < K; ++k) col_sig[(int64_t)i * K + k] = SIG[((int64_t)i * K + k) * S + s];
        total += oracle_color_relaxed_conflicts(n, K, rp, col, col_sig) + gamma * oracle_color_entropy(n, K, col_sig, P->a_ent);
    }
    if (P->alpha_comm != 0.0)
        for (int32_t i = 0; i < n; ++i)
            for (int32_t k = 0; k < K; ++k) {
                double mean, std;
                color_stats(SIG, K, S, i, k, P->comm_eps, &mean, &std);
                total -= (double)S * P->alpha_comm * std;
            }
    free(SIG);
    free(col_sig);
    return total;
}

/*
 * dR/dW at W (interior of [0,1]): with g_ik = dR/dsigma_ik =
 *   sum_{j in N(i)} sigma_jk                        (relaxed conflicts)
 *   + gamma (-c_K a K (K sigma_ik - 1)^(a-1))       (entropy)
 *   - alpha (sigma_ik - mean_ik) / STD_ik            (communication, per replica)
 * the Clamp-normalise Jacobian d sigma_ik' / d W_ik = (delta_kk' - sigma_ik') / sum_k W
 * gives dR/dW_ik = (g_ik - sum_k' sigma_ik' g_ik') / sum_k W (0 for a zero row).
 * G and Gs (sum of absolute contributions, same propagation) are [n][K][S].
 */
void oracle_color_gradient(const oracle_params *P, int32_t n, int32_t K, const int32_t *rp, const int32_t *col,
                           double gamma, const double *W, double *G, double *Gs)
{
    int32_t S = P->S;
    size_t NKS = (size_t)n * (size_t)K * (size_t)S;
    double *SIG = (double *)malloc(sizeof(double) * (NKS ? NKS : 1));
    color_sigma_all(n, K, S, W, SIG);
    double cK = color_cK(K, P->a_ent);
    #pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < n; ++i) {
        double *gs = (double *)malloc(sizeof(double) * (size_t)K);
        double *as = (double *)malloc(sizeof(double) * (size_t)K);
        double *mean = (double *)malloc(sizeof(double) * (size_t)K);
        double *std = (double *)malloc(sizeof(double) * (size_t)K);
        for (int32_t k = 0; k < K; ++k) color_stats(SIG, K, S, i, k, P->comm_eps, &mean[k], &std[k]);
        for (int32_t s = 0; s < S; ++s) {
            double wsum = 0.0;
            for (int32_t k = 0; k < K; ++k) wsum += W[((int64_t)i * K + k) * S + s];
            double dot = 0.0, adot = 0.0;
            for (int32_t k = 0; k < K; ++k) {
                double sig = SIG[((int64_t)i * K + k) * S + s];
                double y = 0.0;
                for (int32_t e = rp[i]; e < rp[i + 1]; ++e) y += SIG[((int64_t)col[e] * K + k) * S + s];
                double ent = gamma * (-cK * (double)P->a_ent * (double)K * ipow((double)K * sig - 1.0, P->a_ent - 1));
                double comm = P->alpha_comm != 0.0 ? -P->alpha_comm * (sig - mean[k]) / std[k] : 0.0;
                gs[k] = y + ent + comm;
                /* scale of the communication term: sigma and its mean are rounded before
                   they are subtracted, as in the binary gradient's scale */
                double comm_scale = P->alpha_comm != 0.0 ? P->alpha_comm * (fabs(sig) + fabs(mean[k])) / std[k] : 0.0;
                as[k] = fabs(y) + fabs(ent) + comm_scale;
                dot += sig * gs[k];
                adot += sig * as[k];
            }
            for (int32_t k = 0; k < K; ++k) {
                int64_t e = ((int64_t)i * K + k) * S + s;
                G[e] = wsum > 0.0 ? (gs[k] - dot) / wsum : 0.0;
                if (Gs) Gs[e] = wsum > 0.0 ? (as[k] + adot) / wsum : 0.0;
            }
        }
        free(gs); free(as); free(mean); free(std);
    }
    free(SIG);
}

/*
 * One step on W[n][K][S] (in place), as the binary step: AdamW with decoupled
 * decay, + sqrt(2 lr T) xi with xi the Gaussian of counter row i*K + k, then
 * the projection to [0,1]. grad/gabs (optional) receive dR/dW and its scale.
 */
void oracle_color_step(const oracle_params *P, int32_t n, int32_t K, const int32_t *rp, const int32_t *col, int32_t t,
                       double *W, double *m, double *v, double *grad, double *gabs)
{
    int32_t S = P->S;
    size_t NKS = (size_t)n * (size_t)K * (size_t)S;
    double *G = (double *)malloc(sizeof(double) * (NKS ? NKS : 1));
    double *Gs = (double *)malloc(sizeof(double) * (NKS ? NKS : 1));
    oracle_color_gradient(P, n, K, rp, col, oracle_gamma(P, t), W, G, Gs);
    double bc1 = 1.0 - pow(P->beta1, (double)(t + 1));
    double bc2 = 1.0 - pow(P->beta2, (double)(t + 1));
    double noise_scale = sqrt(2.0 * P->lr * P->temperature);
    #pragma omp parallel for schedule(static)
    for (int32_t i = 0; i < n; ++i)
        for (int32_t k = 0; k < K; ++k)
            for (int32_t s = 0; s < S; ++s) {
                int64_t e = ((int64_t)i * K + k) * S + s;
                double g = G[e];
                double wn = W[e] * (1.0 - P->lr * P->weight_decay);
                double mm = P->beta1 * m[e] + (1.0 - P->beta1) * g;
                double vv = P->beta2 * v[e] + (1.0 - P->beta2) * g * g;
                wn -= (P->lr / bc1) * mm / (sqrt(vv) / sqrt(bc2) + P->adam_eps);
                if (noise_scale != 0.0) wn += noise_scale * oracle_gaussian(P->seed, i * K + k, s, t);
                if (wn < 0.0) wn = 0.0;
                if (wn > 1.0) wn = 1.0;
                W[e] = wn;
                m[e] = mm;
                v[e] = vv;
                if (grad) grad[e] = g;
                if (gabs) gabs[e] = Gs[e];
            }
    free(G);
    free(Gs);
}

/* initial W: U(0,1] of counter row i*K + k (tag 0) */
void oracle_color_init(int32_t n, int32_t K, int32_t S, uint64_t seed, double *W)
{
    for (int32_t i = 0; i < n; ++i)
        for (int32_t k = 0; k < K; ++k)
            for (int32_t s = 0; s < S; ++s) W[((int64_t)i * K + k) * S + s] = oracle_uniform(seed, i * K + k, s, 0, 0);
}

/* rounding x_is = argmax_k sigma_iks (ties -> lowest k) and the conflicts of every
 * replica; returns the replica with the fewest conflicts (ties -> lowest s) */
int32_t oracle_color_round(int32_t n, int32_t K, int32_t S, const int32_t *rp, const int32_t *col, const double *W,
                           int32_t *x_all, int64_t *conflicts)
{
    int32_t *x = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    double *row = (double *)malloc(sizeof(double) * (size_t)K);
    int32_t best = -1;
    for (int32_t s = 0; s < S; ++s) {
        for (int32_t i = 0; i < n; ++i) {
            color_sigma_row(W, K, S, i, s, row);
            int32_t arg = 0;
            for (int32_t k = 1; k < K; ++k)
                if (row[k] > row[arg]) arg = k;
            x[i] = arg;
            if (x_all) x_all[(int64_t)i * S + s] = arg;
        }
        conflicts[s] = oracle_color_conflicts(n, rp, col, x);
        if (best < 0 || conflicts[s] < conflicts[best]) best = s;
    }
    free(x);
    free(row);
    return best;
}

/* full run: init, P->K steps, final rounding; W_out (optional) gets the final state */
int32_t oracle_color_anneal(const oracle_params *P, int32_t n, int32_t K, const int32_t *rp, const int32_t *col,
                            int32_t steps_to_run, int64_t *conflicts, int32_t *x_all, double *W_out)
{
    int32_t S = P->S;
    size_t NKS = (size_t)n * (size_t)K * (size_t)S;
    double *W = (double *)malloc(sizeof(double) * (NKS ? NKS : 1));
    double *m = (double *)calloc(NKS ? NKS : 1, sizeof(double));
    double *v = (double *)calloc(NKS ? NKS : 1, sizeof(double));
    oracle_color_init(n, K, S, P->seed, W);
    int32_t steps = steps_to_run >= 0 ? steps_to_run : P->K;
    for (int32_t t = 0; t < steps; ++t) oracle_color_step(P, n, K, rp, col, t, W, m, v, NULL, NULL);
    int32_t best = oracle_color_round(n, K, S, rp, col, W, x_all, conflicts);
    if (W_out) memcpy(W_out, W, sizeof(double) * NKS);
    free(W); free(m); free(v);
    return best;
}

int32_t oracle_num_threads(void)
{
#ifdef _OPENMP
    return (int32_t)omp_get_max_threads();
#else
    return 1;
#endif
}
