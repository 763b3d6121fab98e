/*
 * grape_oracle.c - plain FP64 CPU oracle of open GRAPE with RK4 propagation
 * (arXiv:1609.03170).  TEST INFRASTRUCTURE ONLY: called from the tests, the
 * smoke check and the CPU baseline of bench.py through oracle/sparse.py.
 * It shares no code with the CUDA path.
 *
 * The steps follow the paper's notation:
 *   L rho   = -i[H, rho] + sum_j gamma_j (a_j rho a_j^+ - {a_j^+ a_j, rho}/2)
 *             (Eq. master, Eq. disspation)
 *   L^+ X   = i[H, X] + sum_j gamma_j (a_j^+ X a_j - {a_j^+ a_j, X}/2)
 *             (dual under the bilinear pairing Tr(X rho))
 *   H_j     = H_0 + sum_k u_k(j) H_k                      (Eq. Hamiltonian)
 *   forward: slice by slice, n_RK classic RK4 substeps of h = (T/N)/n_RK,
 *            rho_j saved after every slice                (Sec. 3, Eq. rkmaster)
 *   cost:    Phi = sum_s Re Tr(sigma rho_s(T))            (Eq. phi, Eq. Phi0)
 *   mode 1:  exact discrete adjoint: reverse mode through the four RK4 stages
 *            of every substep, each stage adding Re Tr(kb_s (-i)[H_k, y_s])
 *   mode 2:  the paper's first-order gradient (Eq. dphidu)
 *            Re(-i dt Tr(lambda_j [H_k, rho_j])), lambda from backward RK4
 *            on L^+ starting at lambda_N = sigma (Sec. 3 backward integration)
 *   mode 0:  forward and cost only.
 * Two variants of the paper: a control k may drive the rate of dissipator j
 * (rate gamma_j u_k(j) in slice j, dL/du_k = gamma_j D[a_j]; the remarks after
 * Eq. partialuk), and a running cost -beta dt sum_{n=0..N} Tr(A rho_n) with A
 * diagonal (Sec. 5 and App. B, the photon-number penalty) adds -beta dt A to
 * the adjoint at the final time and after every backward slice.
 *
 * Operators are sparse coordinate lists: op 0 = H_0, ops 1..R = H_k,
 * ops R+1..R+J = a_j.  Matrices are d x d row-major, complex values stored as
 * interleaved (re, im) doubles.  Initial states are independent, so an OpenMP
 * loop runs over them; their contributions are added in state order.
 */
#include <complex.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double _Complex cplx;

typedef struct {
    int nnz;
    int *r, *c;
    cplx *v;
} sparse;

/* Y += s A X */
static void left(const sparse *A, cplx s, const cplx *X, cplx *Y, int d) {
    for (int t = 0; t < A->nnz; t++) {
        cplx v = s * A->v[t];
        const cplx *x = X + (size_t)A->c[t] * d;
        cplx *y = Y + (size_t)A->r[t] * d;
        for (int j = 0; j < d; j++) y[j] += v * x[j];
    }
}

/* Y += s A^+ X   ((A^+)[c][r] = conj(A[r][c])) */
static void left_adj(const sparse *A, cplx s, const cplx *X, cplx *Y, int d) {
    for (int t = 0; t < A->nnz; t++) {
        cplx v = s * conj(A->v[t]);
        const cplx *x = X + (size_t)A->r[t] * d;
        cplx *y = Y + (size_t)A->c[t] * d;
        for (int j = 0; j < d; j++) y[j] += v * x[j];
    }
}

/* Y += s X A */
static void right(const sparse *A, cplx s, const cplx *X, cplx *Y, int d) {
    for (int t = 0; t < A->nnz; t++) {
        cplx v = s * A->v[t];
        int r = A->r[t], c = A->c[t];
        for (int i = 0; i < d; i++) Y[(size_t)i * d + c] += X[(size_t)i * d + r] * v;
    }
}

/* Y += s X A^+ */
static void right_adj(const sparse *A, cplx s, const cplx *X, cplx *Y, int d) {
    for (int t = 0; t < A->nnz; t++) {
        cplx v = s * conj(A->v[t]);
        int r = A->r[t], c = A->c[t];
        for (int i = 0; i < d; i++) Y[(size_t)i * d + r] += X[(size_t)i * d + c] * v;
    }
}

typedef struct {
    int d, R, J;
    sparse H0, *Hc, *jump, *jdj; /* jdj[m] = a_m^+ a_m */
    const double *rate;
    const int *jctl;             /* NULL or [J]: control driving the rate of jump m, -1 none */
    const double *pen;           /* NULL or [d]: diagonal of the running-cost operator A */
    double beta;                 /* its weight */
} model;

/* the slice's generator: H_j and the effective rates */
typedef struct {
    sparse H;
    double *g;
} slice_op;

static void set_zero(cplx *X, size_t n) { memset(X, 0, n * sizeof(cplx)); }

/* a^+ a as a sparse list, through a dense scratch matrix */
static sparse dagger_times(const sparse *a, int d) {
    cplx *D = calloc((size_t)d * d, sizeof(cplx));
    for (int t = 0; t < a->nnz; t++)
        for (int u = 0; u < a->nnz; u++)
            if (a->r[t] == a->r[u])           /* (a^+ a)[c_t][c_u] += conj(a[r][c_t]) a[r][c_u] */
                D[(size_t)a->c[t] * d + a->c[u]] += conj(a->v[t]) * a->v[u];
    sparse s = {0, 0, 0, 0};
    for (size_t i = 0; i < (size_t)d * d; i++) if (D[i] != 0) s.nnz++;
    s.r = malloc(sizeof(int) * (s.nnz + 1));
    s.c = malloc(sizeof(int) * (s.nnz + 1));
    s.v = malloc(sizeof(cplx) * (s.nnz + 1));
    int n = 0;
    for (int i = 0; i < d; i++)
        for (int j = 0; j < d; j++)
            if (D[(size_t)i * d + j] != 0) { s.r[n] = i; s.c[n] = j; s.v[n] = D[(size_t)i * d + j]; n++; }
    free(D);
    return s;
}

/* H_j = H_0 + sum_k u_k H_k as one coordinate list */
static sparse slice_hamiltonian(const model *m, const double *uj) {
    int nnz = m->H0.nnz;
    for (int k = 0; k < m->R; k++) nnz += m->Hc[k].nnz;
    sparse H;
    H.nnz = nnz;
    H.r = malloc(sizeof(int) * (nnz + 1));
    H.c = malloc(sizeof(int) * (nnz + 1));
    H.v = malloc(sizeof(cplx) * (nnz + 1));
    int n = 0;
    for (int t = 0; t < m->H0.nnz; t++, n++) { H.r[n] = m->H0.r[t]; H.c[n] = m->H0.c[t]; H.v[n] = m->H0.v[t]; }
    for (int k = 0; k < m->R; k++)
        for (int t = 0; t < m->Hc[k].nnz; t++, n++) {
            H.r[n] = m->Hc[k].r[t]; H.c[n] = m->Hc[k].c[t]; H.v[n] = uj[k] * m->Hc[k].v[t];
        }
    return H;
}

static void free_sparse(sparse *s) { free(s->r); free(s->c); free(s->v); }

static slice_op slice_operator(const model *m, const double *uj) {
    slice_op S;
    S.H = slice_hamiltonian(m, uj);
    S.g = malloc(sizeof(double) * (m->J + 1));
    for (int j = 0; j < m->J; j++)
        S.g[j] = m->rate[j] * ((m->jctl && m->jctl[j] >= 0) ? uj[m->jctl[j]] : 1.0);
    return S;
}

static void free_slice(slice_op *S) { free_sparse(&S->H); free(S->g); }

/* out = L rho (Eq. master) */
static void lindblad(const model *m, const slice_op *S, const cplx *rho, cplx *out, cplx *tmp) {
    int d = m->d;
    size_t n = (size_t)d * d;
    const sparse *H = &S->H;
    set_zero(out, n);
    left(H, -I, rho, out, d);
    right(H, I, rho, out, d);
    for (int j = 0; j < m->J; j++) {
        double g = S->g[j];
        set_zero(tmp, n);
        left(&m->jump[j], 1.0, rho, tmp, d);
        right_adj(&m->jump[j], g, tmp, out, d);
        left(&m->jdj[j], -0.5 * g, rho, out, d);
        right(&m->jdj[j], -0.5 * g, rho, out, d);
    }
}

/* out = L^+ X */
static void lindblad_dual(const model *m, const slice_op *S, const cplx *X, cplx *out, cplx *tmp) {
    int d = m->d;
    size_t n = (size_t)d * d;
    const sparse *H = &S->H;
    set_zero(out, n);
    left(H, I, X, out, d);
    right(H, -I, X, out, d);
    for (int j = 0; j < m->J; j++) {
        double g = S->g[j];
        set_zero(tmp, n);
        left_adj(&m->jump[j], 1.0, X, tmp, d);
        right(&m->jump[j], g, tmp, out, d);
        left(&m->jdj[j], -0.5 * g, X, out, d);
        right(&m->jdj[j], -0.5 * g, X, out, d);
    }
}

typedef void (*rhs_fn)(const model *, const slice_op *, const cplx *, cplx *, cplx *);

/* one classic RK4 step y -> ynew; optionally keeps the four stage inputs */
static void rk4(rhs_fn f, const model *m, const slice_op *H, double h, const cplx *y,
                cplx *ynew, cplx *stage_in /* 4*n or NULL */, cplx *w /* 6*n work */) {
    size_t n = (size_t)m->d * m->d;
    cplx *k1 = w, *k2 = w + n, *k3 = w + 2 * n, *k4 = w + 3 * n, *yt = w + 4 * n, *tmp = w + 5 * n;
    if (stage_in) memcpy(stage_in, y, n * sizeof(cplx));
    f(m, H, y, k1, tmp);
    for (size_t i = 0; i < n; i++) yt[i] = y[i] + (h / 2) * k1[i];
    if (stage_in) memcpy(stage_in + n, yt, n * sizeof(cplx));
    f(m, H, yt, k2, tmp);
    for (size_t i = 0; i < n; i++) yt[i] = y[i] + (h / 2) * k2[i];
    if (stage_in) memcpy(stage_in + 2 * n, yt, n * sizeof(cplx));
    f(m, H, yt, k3, tmp);
    for (size_t i = 0; i < n; i++) yt[i] = y[i] + h * k3[i];
    if (stage_in) memcpy(stage_in + 3 * n, yt, n * sizeof(cplx));
    f(m, H, yt, k4, tmp);
    for (size_t i = 0; i < n; i++) ynew[i] = y[i] + (h / 6) * (k1[i] + 2 * k2[i] + 2 * k3[i] + k4[i]);
}

/* Tr(A B), bilinear */
static cplx trace_prod(const cplx *A, const cplx *B, int d) {
    cplx s = 0;
    for (int i = 0; i < d; i++)
        for (int j = 0; j < d; j++) s += A[(size_t)i * d + j] * B[(size_t)j * d + i];
    return s;
}

/* Re Tr(Kb (dL/du_k) Y): (-i)[H_k, Y], plus gamma_j D[a_j] Y for every
   dissipator j whose rate control k drives */
static double control_term(const model *m, int k, const cplx *Kb, const cplx *Y, cplx *tmp) {
    int d = m->d;
    size_t n = (size_t)d * d;
    set_zero(tmp, n);
    left(&m->Hc[k], -I, Y, tmp, d);
    right(&m->Hc[k], I, Y, tmp, d);
    if (m->jctl) {
        cplx *t2 = malloc(sizeof(cplx) * n);
        for (int j = 0; j < m->J; j++) {
            if (m->jctl[j] != k) continue;
            double g = m->rate[j];
            set_zero(t2, n);
            left(&m->jump[j], 1.0, Y, t2, d);
            right_adj(&m->jump[j], g, t2, tmp, d);
            left(&m->jdj[j], -0.5 * g, Y, tmp, d);
            right(&m->jdj[j], -0.5 * g, Y, tmp, d);
        }
        free(t2);
    }
    return creal(trace_prod(Kb, tmp, d));
}

/* Re Tr(A X) for the diagonal A; and X += s A */
static double pen_value(const model *m, const cplx *X) {
    double t = 0;
    for (int i = 0; i < m->d; i++) t += m->pen[i] * creal(X[(size_t)i * m->d + i]);
    return t;
}
static void add_pen(const model *m, double s, cplx *X) {
    for (int i = 0; i < m->d; i++) X[(size_t)i * m->d + i] += s * m->pen[i];
}

static void one_state(const model *m, int n_slices, int n_rk, double T, const double *u,
                      const cplx *rho0, const cplx *sig, int mode,
                      double *F, double *G /* n_slices*R, zeroed */, cplx *rhoT) {
    int d = m->d, R = m->R;
    size_t n = (size_t)d * d;
    double dt = T / n_slices, h = dt / n_rk;
    int keep = (mode != 0);
    cplx *traj = malloc(sizeof(cplx) * n * (keep ? (size_t)n_slices + 1 : 2));
    cplx *w = malloc(sizeof(cplx) * n * 6);
    memcpy(traj, rho0, n * sizeof(cplx));
    cplx *cur = traj;
    double pen_sum = m->pen ? pen_value(m, cur) : 0.0;    /* boundary n = 0 */
    for (int j = 0; j < n_slices; j++) {
        slice_op H = slice_operator(m, u + (size_t)j * R);
        cplx *nxt = keep ? traj + (size_t)(j + 1) * n : traj + (size_t)((j + 1) & 1) * n;
        const cplx *y = cur;
        for (int r = 0; r < n_rk; r++) {
            rk4(lindblad, m, &H, h, y, nxt, NULL, w);
            y = nxt;
        }
        cur = nxt;
        if (m->pen) pen_sum += pen_value(m, cur);          /* boundary j + 1 */
        free_slice(&H);
    }
    *F = creal(trace_prod(sig, cur, d)) - m->beta * dt * pen_sum;
    if (rhoT) memcpy(rhoT, cur, n * sizeof(cplx));

    if (mode == 1) {
        cplx *mu = malloc(sizeof(cplx) * n);
        cplx *st = malloc(sizeof(cplx) * n * 4 * (size_t)n_rk);
        cplx *ys = malloc(sizeof(cplx) * n * 2);
        cplx *kb = malloc(sizeof(cplx) * n), *yb = malloc(sizeof(cplx) * n * 4);
        cplx *tmp = malloc(sizeof(cplx) * n), *tmp2 = malloc(sizeof(cplx) * n);
        memcpy(mu, sig, n * sizeof(cplx));
        if (m->pen) add_pen(m, -m->beta * dt, mu);
        for (int j = n_slices - 1; j >= 0; j--) {
            slice_op H = slice_operator(m, u + (size_t)j * R);
            /* stage inputs of the slice, recomputed from the saved rho_j */
            const cplx *y = traj + (size_t)j * n;
            for (int r = 0; r < n_rk; r++) {
                cplx *yo = ys + (size_t)(r & 1) * n;
                rk4(lindblad, m, &H, h, y, yo, st + (size_t)r * 4 * n, w);
                y = yo;
            }
            for (int r = n_rk - 1; r >= 0; r--) {
                const cplx *Y = st + (size_t)r * 4 * n;   /* y1..y4 */
                double coef_mu[4] = {h / 6, h / 3, h / 3, h / 6};
                double coef_yb[4] = {h / 2, h / 2, h, 0.0};  /* kb_s += coef * yb_{s+1} */
                for (int s = 3; s >= 0; s--) {
                    for (size_t i = 0; i < n; i++)
                        kb[i] = coef_mu[s] * mu[i] + (s < 3 ? coef_yb[s] * yb[(size_t)(s + 1) * n + i] : 0.0);
                    lindblad_dual(m, &H, kb, yb + (size_t)s * n, tmp);
                    for (int k = 0; k < R; k++)
                        G[(size_t)j * R + k] += control_term(m, k, kb, Y + (size_t)s * n, tmp2);
                }
                for (size_t i = 0; i < n; i++)
                    mu[i] += yb[i] + yb[n + i] + yb[2 * n + i] + yb[3 * n + i];
            }
            if (m->pen) add_pen(m, -m->beta * dt, mu);      /* running cost at boundary j */
            free_slice(&H);
        }
        free(mu); free(st); free(ys); free(kb); free(yb); free(tmp); free(tmp2);
    } else if (mode == 2) {
        cplx *lam = malloc(sizeof(cplx) * n), *lam2 = malloc(sizeof(cplx) * n);
        cplx *tmp = malloc(sizeof(cplx) * n);
        memcpy(lam, sig, n * sizeof(cplx));
        if (m->pen) add_pen(m, -m->beta * dt, lam);
        for (int j = n_slices; j >= 1; j--) {
            const cplx *rho_j = traj + (size_t)j * n;
            for (int k = 0; k < R; k++) {
                /* Re(-i dt Tr(lambda_j [H_k, rho_j])) = dt * Re Tr(lambda_j (-i)[H_k, rho_j]) */
                G[(size_t)(j - 1) * R + k] += dt * control_term(m, k, lam, rho_j, tmp);
            }
            slice_op H = slice_operator(m, u + (size_t)(j - 1) * R);
            for (int r = 0; r < n_rk; r++) {
                rk4(lindblad_dual, m, &H, h, lam, lam2, NULL, w);
                memcpy(lam, lam2, n * sizeof(cplx));
            }
            if (m->pen) add_pen(m, -m->beta * dt, lam);
            free_slice(&H);
        }
        free(lam); free(lam2); free(tmp);
    }
    free(traj);
    free(w);
}

static sparse view(const int *op_ptr, const int *rows, const int *cols, const double *vals, int o) {
    sparse s;
    int a = op_ptr[o], b = op_ptr[o + 1];
    s.nnz = b - a;
    s.r = malloc(sizeof(int) * (s.nnz + 1));
    s.c = malloc(sizeof(int) * (s.nnz + 1));
    s.v = malloc(sizeof(cplx) * (s.nnz + 1));
    for (int t = 0; t < s.nnz; t++) {
        s.r[t] = rows[a + t];
        s.c[t] = cols[a + t];
        s.v[t] = vals[2 * (a + t)] + I * vals[2 * (a + t) + 1];
    }
    return s;
}

int grape_oracle_run(int d, int n_states, int n_slices, int n_rk, double T,
                     int n_controls, int n_jumps,
                     const int *op_ptr, const int *rows, const int *cols, const double *vals,
                     const double *rates, const int *jump_control,
                     const double *pen_diag, double pen_beta,
                     const double *rho0, const double *sigma, int sigma_per_state,
                     const double *u, int mode, int n_threads,
                     double *F, double *grad, double *rhoT) {
    if (d <= 0 || n_states <= 0 || n_slices <= 0 || n_rk <= 0 || mode < 0 || mode > 2) return 1;
    model m;
    m.d = d; m.R = n_controls; m.J = n_jumps; m.rate = rates;
    m.jctl = jump_control; m.pen = pen_diag; m.beta = pen_beta;
    m.H0 = view(op_ptr, rows, cols, vals, 0);
    m.Hc = malloc(sizeof(sparse) * (n_controls + 1));
    m.jump = malloc(sizeof(sparse) * (n_jumps + 1));
    m.jdj = malloc(sizeof(sparse) * (n_jumps + 1));
    for (int k = 0; k < n_controls; k++) m.Hc[k] = view(op_ptr, rows, cols, vals, 1 + k);
    for (int j = 0; j < n_jumps; j++) {
        m.jump[j] = view(op_ptr, rows, cols, vals, 1 + n_controls + j);
        m.jdj[j] = dagger_times(&m.jump[j], d);
    }
    size_t n = (size_t)d * d;
    size_t gsz = (size_t)n_slices * n_controls;
    double *Fs = calloc(n_states, sizeof(double));
    double *Gs = calloc(gsz * n_states + 1, sizeof(double));
#ifdef _OPENMP
    if (n_threads > 0) omp_set_num_threads(n_threads);
#pragma omp parallel for schedule(static, 1)
#endif
    for (int s = 0; s < n_states; s++) {
        one_state(&m, n_slices, n_rk, T, u,
                  (const cplx *)(rho0 + 2 * n * s),
                  (const cplx *)(sigma + (sigma_per_state ? 2 * n * s : 0)),
                  mode, &Fs[s], Gs + gsz * s, rhoT ? (cplx *)(rhoT + 2 * n * s) : NULL);
    }
    double Ft = 0;
    for (int s = 0; s < n_states; s++) Ft += Fs[s];
    *F = Ft;
    if (grad && mode != 0) {
        for (size_t i = 0; i < gsz; i++) {
            double g = 0;
            for (int s = 0; s < n_states; s++) g += Gs[gsz * s + i];
            grad[i] = g;
        }
    }
    free(Fs); free(Gs);
    free_sparse(&m.H0);
    for (int k = 0; k < n_controls; k++) free_sparse(&m.Hc[k]);
    for (int j = 0; j < n_jumps; j++) { free_sparse(&m.jump[j]); free_sparse(&m.jdj[j]); }
    free(m.Hc); free(m.jump); free(m.jdj);
    return 0;
}

int grape_oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
