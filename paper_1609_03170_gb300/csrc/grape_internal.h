// grape_internal.h - kernel argument blocks shared by grape_kernels.cu and
// grape_api.cu.  Not part of the public ABI (include/grape.h is).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#define GRAPE_MAXB 12    // bands of the (effective) Hamiltonian part A
#define GRAPE_MAXT 12    // jump sandwich terms vL[i] conj(vR[j]) X[i+oL][j+oR]
#define GRAPE_MAXR 8     // control Hamiltonians
#define GRAPE_MAXCB 8    // (control, band) pairs seen by the trace kernel
#define GRAPE_MAXDO 8    // distinct band offsets among the control bands
#define GRAPE_MAXST 4    // sandwich terms of dissipators whose rate is a control
#define GRAPE_PROP_THREADS 512   // threads per CTA of the propagation kernel

// One direction of the Lindblad action in the common form
//   W = -i (A X - X A^+) + sum_t vL_t[i] conj(vR_t[j]) X[i + oL_t][j + oR_t]
// Forward (Eq. master):   A = H_eff = H_0 - i/2 sum gamma c^+ c + sum_k u_k H_k,
//                         terms from sqrt(gamma) c_m (all band pairs).
// Dual (adjoint):         A = -H_eff^+, terms from sqrt(gamma) c_m^+.
// A(u) = A0 + sum_k u_k Ak is rebuilt in shared memory once per slice.
struct PropTables {
    int nb, nt;
    int nbr;                    // the first nbr bands are real for every control value
                                // (real multiply-adds); the offset-0 band is never among them
    int off[GRAPE_MAXB];        // band offsets o_b: A_b[i] = A[i][i + o_b]
    int off_row[GRAPE_MAXB];    // o_b * d (flat shift of row i -> i + o_b)
    int jflat[GRAPE_MAXT];      // oL_t * d + oR_t
    int joL[GRAPE_MAXT];        // oL_t
    int joR[GRAPE_MAXT];        // oR_t
    int b0;                     // index of the offset-0 band, -1 if none
    int jdiag;                  // bit t set: jump term t has oL_t = oR_t = 0
    int jrate;                  // bit t set: jump term t is scaled by a control (its rate is a control)
    int jctl[GRAPE_MAXT];       // that control, -1: fixed
    const void *A0s;            // [nb][d], the kernels' storage format
    const void *Aks;            // [R][nb][d], the kernels' storage format
    const double2 *vL;          // [nt][d]
    const double2 *vR;          // [nt][d]
    const void *vLs, *vRs;      // the same in the kernels' storage format (read from global
                                // memory by the grid kernel)
};

// One RK4 sweep over substeps [sub_begin, sub_end) of one segment.  The
// per-substep recurrence for a base value x (rho forward, mu adjoint) is
//   z_0 = g0 x;  for s = 0..3:  w_s = Op(z_s);  acc += a_s w_s;
//                               z_{s+1} = g_{s+1} x + b_{s+1} w_s
//   x <- acc (acc starts at x)
// which is classic RK4 forward (g = 1, a = h(1/6,1/3,1/3,1/6),
// b = h(-,1/2,1/2,1)) and its exact reverse-mode adjoint backward
// (g = h(1/6,1/3,1/3,1/6), a = 1, b = h(-,1,1/2,1/2)).
struct PropArgs {
    PropTables tab;
    int d, R, n_states;
    int ncl, chunk, halo, win, reach;   // cluster split of the d*d matrix
    const double *u;                    // [n_slices][R]
    int n_rk;
    long long sub_begin, sub_end;       // substep range
    int reverse;
    double g[4], a[4], b[4];
    int store_map[4];                   // stage s -> slot of the stage store
    // state buffers are in the kernel's storage format (16 bytes per complex
    // entry: double2 for FP64, float4 hi/lo pairs for double-float)
    const void *x_in;                   // [n_states][d*d]
    void *x_out;                        // [n_states][d*d] (may alias x_in)
    void *stage_store;                  // [(n - sub_begin)][4][n_states][d(d+1)/2] or null: every
                                        // stage input, packed upper triangle (row-major order)
    void *bound_store;                  // [slot][n_states][d*d] or null
    long long bound_step;               // substeps between bound stores
    // Hermitian kernel (upper triangle only): the cluster's ownership and
    // window tables, see GRAPE_HTAB_* below
    const int *htab;
    int htab_len;                       // ints in htab
    int hb;                             // stored half-band below the diagonal
    int cu;                             // upper-triangle entries per CTA
    int maxwin;                         // largest window (entries) of the cluster
    int rt_rows;                        // rows of the largest push table
    int fold;                           // Hermitian kernel: own-entry coefficients folded (D table)
    int jcache;                         // Hermitian kernel, real jump tables: coefficients of the
                                        // jump terms cached per owned entry
    int defer;                          // Hermitian kernel: next values kept until the cluster
                                        // wait before the pushes (hides its latency)
    const double *src;                  // adjoint source on the diagonal per row (App. B), or null
    // grid kernel (stage values in global memory, windows loaded per stage;
    // ncl = CTAs per state, htab/maxwin/cu/hb as for the Hermitian kernel)
    void *gbuf;                         // [2][n_states][d*d] stage-input buffers
    unsigned *gbar;                     // [2]: error word, 1 a grid kernel wait gave up, 2 a
                                        // window wait of the Hermitian kernel gave up
    unsigned *gflag;                    // [n_states][ncl] finished push rounds per CTA (zeroed
                                        // before every launch)
    const int *ntab;                    // [ncl][ntab_stride]: count and ranks of a CTA's neighbours
    int ntab_stride;
    long long spin_limit;               // polls of a grid-kernel wait before it gives up
};

#define GRAPE_GRID_THREADS 512

// Layout of the Hermitian kernel's table (ints), for a cluster of ncl CTAs:
//   [4k + 0..3]            u0, u1 (owned upper-triangle range), wr0, nrows of CTA k
//   [4 ncl + k]            start of CTA k's row-offset list (k = 0..ncl)
//   [row-offset lists]     CTA k: nrows_k + 1 cumulative window offsets
//   [kfirst[d], klast[d]]  first and last CTA whose window holds row r
#define GRAPE_HTAB_CTA(k) (4 * (k))
#define GRAPE_HTAB_LISTS(ncl) (4 * (ncl))

// Trace products of the gradient (Eq. dphidu), per output row j:
//   G[j][k] = weight * sum_q (-2) Im sum_b sum_m Hk_b[m] P_{o_b}[m],
//   P_o[m]  = sum_l K_q[m + o][l] conj(Y_q[m][l]),
// i.e. -2 Im Tr(K Y H_k) = Re Tr(K (-i)[H_k, Y]) for Hermitian K and Y.
// Packed storage (exact gradient): K_q and Y_q hold upper triangles
// (d(d+1)/2 entries, row-major), and the same sum runs over the upper
// entries (i, j), j >= i, as
//   Tr(K Y H) = sum_{i<=j} sum_o [ H_o[i] conj(Y_ij) K_{i+o,j}
//                                  + (i < j) H_o[j] Y_ij conj(K_{i,j+o}) ]
// (H_o[m] = H[m][m+o]; an entry below the diagonal is the conjugate of its
// mirror).  Each row's pairs are split by state and by chunks of entries.
struct TraceArgs {
    int d, R;
    int ncb, ndo;
    int cb_k[GRAPE_MAXCB];      // control of band entry c
    int cb_do[GRAPE_MAXCB];     // distinct-offset index of band entry c
    int do_off[GRAPE_MAXDO];    // distinct offsets
    const void *cb_s;           // [ncb][d]  Hk_b[m], storage format of the number type
    const void *K;              // adjoint-side matrices (storage format)
    const void *Y;              // forward-side matrices (storage format)
    long long npairs;           // matrices per output row
    int n_rows;
    double weight;
    double *G;                  // [n_rows][R]
    // nsplit > 1: each row's pairs are split over nsplit CTAs writing
    // part[row][split][R]; trace_finish_kernel adds the splits in order
    int nsplit;
    double *part;
    // packed storage: nsplit = n_states * nchunk CTAs per row, CTA (state s,
    // chunk c) sums the entries [c * 256 * epc, (c + 1) * 256 * epc) of state
    // s over its pairs q = (substep * 4 + stage) * n_states + s
    int packed, nchunk, epc, n_states;
    // controls on dissipation rates: the sandwich part of Re Tr(kb D[c] y),
    // sum over m, l of conj(K[m][l]) vL[m] conj(vR[l]) Y[m+oL][l+oR] per term
    int nst;
    int st_k[GRAPE_MAXST];
    int st_oL[GRAPE_MAXST], st_oR[GRAPE_MAXST];
    const void *st_vLs, *st_vRs;    // [nst][d], storage format
    // staged trace (packed storage, nst == 0, ndo <= 4): per 256-entry block
    // b of the packed triangle, the runs of K its entries' neighbours fall in
    // are copied to shared memory with Y's block, per pair, into nbuf buffers
    // of 256 + kcap entries
    int tile, kcap, nbuf;
    const int4 *tblk;               // [blocks]: first run, run count, K entries copied
    const int4 *trun;               // runs: packed start, length, offset in the buffer's K part
    const uint4 *tnb;               // [NU]: per distinct offset (i+o, j) and (i, j+o) as 16-bit
                                    // buffer indices (bit 15: conjugate of the mirror; 0xffff: none)
    const unsigned *tij;            // [NU]: i | j << 16 of packed entry u
    unsigned *err;                  // error word: 3 when a copy wait gave up
    long long spin;                 // SM cycles a copy wait may take (0: give up at once)
};

// dynamic shared memory of the staged trace kernel: 8 mbarriers, the
// per-band sums [8][256] (16 B each), nbuf buffers of 256 + kcap entries
inline size_t trace_tile_smem(int nbuf, int kcap) {
    return 64 + (size_t)GRAPE_MAXCB * 256 * 16 + (size_t)nbuf * (256 + kcap) * 16;
}

// Launchers, one set per number type: _f64 native FP64, _df double-float.
#define GRAPE_DECLARE_LAUNCHERS(SUFFIX)                                                        \
    cudaError_t grape_launch_prop_##SUFFIX(const PropArgs &p, int threads, int variant,         \
                                           size_t smem, cudaStream_t stream);                   \
    cudaError_t grape_prepare_prop_##SUFFIX(int variant, size_t smem, int ncl);                \
    cudaError_t grape_max_active_clusters_##SUFFIX(int threads, int variant, size_t smem,       \
                                                   int ncl, int n_blocks, int *clusters);      \
    cudaError_t grape_launch_trace_##SUFFIX(const TraceArgs &p, cudaStream_t stream);          \
    cudaError_t grape_launch_trace_finish_##SUFFIX(const TraceArgs &p, cudaStream_t stream);   \
    cudaError_t grape_launch_cost_##SUFFIX(const void *rho, const void *sigma, int n_states,    \
                                           int d2, double *F, cudaStream_t stream);             \
    cudaError_t grape_launch_to_double_##SUFFIX(const void *src, double2 *dst, size_t n,        \
                                                cudaStream_t stream);                           \
    cudaError_t grape_launch_grid_##SUFFIX(const PropArgs &p, int nblocks, int variant,         \
                                           size_t smem, cudaStream_t stream);                   \
    cudaError_t grape_prepare_grid_##SUFFIX(int variant, size_t smem_total, size_t smem,        \
                                            int *max_blocks);                                  \
    cudaError_t grape_launch_add_diag_##SUFFIX(void *x, const double *src, int d, int n_states, \
                                               cudaStream_t stream);                            \
    cudaError_t grape_launch_penalty_rows_##SUFFIX(const void *x, long long row_stride, int rows, \
                                                   int n_states, int d, const double *diag,     \
                                                   double *out, int packed, cudaStream_t stream); \
    cudaError_t grape_launch_penalty_finish_##SUFFIX(const double *pen, long long count,        \
                                                     double scale, double *F, cudaStream_t stream);

GRAPE_DECLARE_LAUNCHERS(f64)
GRAPE_DECLARE_LAUNCHERS(df)

// ---------------------------------------------------------------------------
// Device state of one projected L-BFGS optimisation (serving loop).
struct LbfgsState {
    double f;        // objective -Phi at the accepted point
    double step;     // step multiplier along the L-BFGS direction
    double gamma;    // s.y / y.y of the newest curvature pair
    double pgnorm;   // max-norm of the projected gradient at the accepted point
    int evals;       // gradient evaluations consumed
    int accepted;    // accepted points
    int hist;        // stored curvature pairs
    int head;        // next ring slot
    int status;      // 0 running, 1 evaluation budget used, 2 converged or stalled
    int pad;
};

struct LbfgsArgs {
    LbfgsState *state;
    int n, m, max_evals;
    double u_min, u_max, tol, step0;
    const double *F, *G;                         // gradient evaluation at ut
    double *u, *g, *ut, *dir, *S, *Y, *rho, *alpha;
};

cudaError_t grape_launch_lbfgs(const LbfgsArgs &a, cudaStream_t s);

// Gaussian control filter (App. A): `in` -> `out`, row-major [index][control];
// forward: N controls -> M subpixels, adjoint: M subpixel gradients -> N.
struct FilterArgs {
    int N, M, R;
    double Dt, dt;                      // control and subpixel lengths
    double w0[GRAPE_MAXR];              // reference bandwidth per control
    const double *in;
    double *out;
};
cudaError_t grape_launch_filter(const FilterArgs &a, bool adjoint, cudaStream_t s);

// FMA throughput of the current device (grape_probe.cu): TFLOP/s (two flops
// per multiply-add) of the FP32 pipes (GRAPE_PREC_DF64) or the FP64 pipe
// (GRAPE_PREC_FP64), and the duration of the timed run.
cudaError_t grape_probe_fma(int precision, double *tflops, double *ms);
