// grape_kernels.cuh - sm_103a kernels of the open-GRAPE hot path, written
// once over the number type (grape_num.cuh) and instantiated for native FP64
// (grape_kernels_f64.cu) and double-float on the FP32 pipes
// (grape_kernels_df.cu).
//
//  prop_h_kernel  RK4 propagation (forward, Sec. 3 Eq. rkmaster, or the exact
//                 adjoint, Eq. lambda) of one density matrix per thread-block
//                 cluster, upper triangle only (every stage value is
//                 Hermitian); the state stays in the cluster's shared memory
//                 as compact row windows, halo values are pushed with st.async
//                 and counted on the receiving window's mbarrier.  The default
//                 kernel; specialised on the band/jump layout (Shape) and on
//                 one entry per thread.
//  prop_kernel    the same over contiguous chunks of the full matrix (when the
//                 Hermitian windows do not fit).
//  prop_g_kernel  the Hermitian kernel's arithmetic over CTAs of the whole
//                 device, for states beyond a cluster's shared memory: stage
//                 values in global memory (L2), row windows loaded per stage,
//                 neighbour-to-neighbour flags with bounded waits.
//  trace_tile_kernel, trace_packed_fast_kernel, trace_packed_kernel
//                 per-slice gradient traces of Eq. (dphidu) on the packed
//                 stage storage (the first stages the operands in shared
//                 memory through a warp-specialised TMA pipeline); fixed
//                 (state, chunk) partials summed in order by
//                 trace_finish_kernel, so no bit depends on the launch.
//  trace_kernel   the first-order gradient's traces on full matrices.
//  cost_kernel    Phi = sum_s Re Tr(sigma_s rho_s(T)) (Eq. phi), fixed order.
//  penalty kernels, add_diag_kernel  the running-cost penalty (App. B).
//  to_double_kernel  storage format -> complex128 (rho(T) output).
#pragma once

#include "grape_internal.h"
#include "grape_num.cuh"

#include <type_traits>

namespace grape_k {

using namespace grape_num;

// Cluster-wide barrier between RK stages.  The per-entry loops before it
// leave warps diverged (the chunk is not a multiple of the block size), so
// the warp is reconverged explicitly and the non-.aligned forms are used,
// which are defined for threads arriving independently.
__device__ __forceinline__ void cluster_sync_all() {
    __syncwarp();
    asm volatile("barrier.cluster.arrive.release;\n\t"
                 "barrier.cluster.wait.acquire;" ::: "memory");
}

// The running cost's source (App. B, photon-number penalty): added to the
// adjoint's diagonal when a backward sweep crosses a slice boundary, i.e.
// after the slice's first substep (n a multiple of n_RK).
template <class Num>
__device__ __forceinline__ typename Num::val with_source(const PropArgs &p, long long n, int i, int j,
                                                         typename Num::val v) {
    if (p.src && p.reverse && (n % p.n_rk) == 0 && i == j)
        return Num::add_real(v, Num::real_const(p.src[i]));
    return v;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ uint32_t map_to_rank(uint32_t addr, uint32_t rank) {
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
__device__ __forceinline__ void st_remote(uint32_t addr, double2 v) {
    asm volatile("st.shared::cluster.v2.f64 [%0], {%1, %2};" ::"r"(addr), "d"(v.x), "d"(v.y)
                 : "memory");
}
__device__ __forceinline__ void st_remote(uint32_t addr, float4 v) {
    asm volatile("st.shared::cluster.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(v.x),
                 "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
}

// A(u_j) = A0 + sum_k u_k(j) Ak in the number type, from tables in its
// storage format: in the double-float build every operation runs on the FP32
// pipes (the slice's R controls are split into float pairs once per CTA, in
// shared memory).  Called by every thread of the CTA (it holds a barrier).
template <class Num>
__device__ __forceinline__ void build_bands(typename Num::store_t *dst, const PropArgs &p,
                                            int slice) {
    using S = typename Num::store_t;
    using R = typename Num::real_t;
    __shared__ R ucv[GRAPE_MAXR];
    const int nbd = p.tab.nb * p.d;
    const double *uj = p.u + (size_t)slice * p.R;
    if (threadIdx.x < p.R) ucv[threadIdx.x] = Num::real_const(__ldg(&uj[threadIdx.x]));
    __syncthreads();
    const S *A0 = static_cast<const S *>(p.tab.A0s);
    const S *Ak = static_cast<const S *>(p.tab.Aks);
    for (int idx = threadIdx.x; idx < nbd; idx += blockDim.x) {
        typename Num::val v = Num::load(A0[idx]);
        for (int k = 0; k < p.R; ++k) v = Num::axpy(ucv[k], Num::load(Ak[(size_t)k * nbd + idx]), v);
        dst[idx] = Num::store(v);
    }
}

// Write stage value z of flat element e into the own window and into every
// neighbour window of the cluster that covers e.
template <class S>
__device__ __forceinline__ void push_value(S *buf, const PropArgs &p, int rank, int e, S z) {
    const int wbase = rank * p.chunk - p.halo;
    buf[e - wbase] = z;
    const int c_lo = max(0, rank - p.reach), c_hi = min(p.ncl - 1, rank + p.reach);
    for (int c = c_lo; c <= c_hi; ++c) {
        if (c == rank) continue;
        const int cb = c * p.chunk - p.halo;
        if (e >= cb && e < cb + p.win)
            st_remote(map_to_rank(smem_u32(&buf[e - cb]), (uint32_t)c), z);
    }
}

// W = Op(z) at element (i, j) of the window `cur` (local flat index le):
//   W = -i (A z - z A^+)[i][j] + sum_t vL_t[i] conj(vR_t[j]) z[i+oL_t][j+oR_t]
// Coefficient of jump term q at entry (i, j): vL_q[i] conj(vR_q[j]), times the
// slice's control value when the term belongs to a dissipator whose rate is a
// control (uj = the slice's controls; fixed terms are untouched).
// Rate-controlled terms exist only in problems that run the complex-table
// kernels (REALJ = false); there the callers branch once per call on
// t.jrate (RATE), so no kernel pays for the scaling it does not use (a
// per-term test let the compiler speculate the FP64 conversion of the
// control value into every iteration).
template <class Num, bool RATE>
__device__ __forceinline__ typename Num::real_t jump_real(const PropTables &t, int q, int i, int j, int d,
                                                          const typename Num::store_t *vL,
                                                          const typename Num::store_t *vR,
                                                          const double *uj) {
    return Num::real_mul(Num::re(Num::load(vL[q * d + i])), Num::re(Num::load(vR[q * d + j])));
}
template <class Num, bool RATE>
__device__ __forceinline__ typename Num::val jump_cplx(const PropTables &t, int q, int i, int j, int d,
                                                       const typename Num::store_t *vL,
                                                       const typename Num::store_t *vR,
                                                       const double *uj) {
    typename Num::val c = Num::mul_conjb(Num::load(vL[q * d + i]), Num::load(vR[q * d + j]));
    if (RATE && ((t.jrate >> q) & 1)) c = Num::scale(Num::real_const(uj[t.jctl[q]]), c);
    return c;
}

// REALJ: the jump tables are real, so each jump coefficient is one real
// product.  Loops run over the problem's band and term counts (kept rolled:
// the pair arithmetic makes every iteration long, and unrolled copies
// overflow the instruction cache).
template <class Num, bool REALJ>
__device__ __forceinline__ typename Num::val lindblad_at(const typename Num::store_t *cur, int le,
                                                         int i, int j, int d, const PropTables &t,
                                                         const typename Num::store_t *A,
                                                         const typename Num::store_t *vL,
                                                         const typename Num::store_t *vR,
                                                         const double *uj) {
    typename Num::acc w = Num::acc_zero();
#pragma unroll 1
    for (int b = 0; b < t.nb; ++b) {
        Num::mac(w, Num::load(A[b * d + i]), Num::load(cur[le + t.off_row[b]]));
        Num::mac_conj_neg(w, Num::load(A[b * d + j]), Num::load(cur[le + t.off[b]]));
    }
    w = Num::acc_minus_i(w);                     // -i (A z - z A^+)
    auto jumps = [&](auto rate) {
        constexpr bool RT = decltype(rate)::value;
#pragma unroll 1
        for (int q = 0; q < t.nt; ++q) {
            if (REALJ)
                Num::mac_real(w, jump_real<Num, RT>(t, q, i, j, d, vL, vR, uj), Num::load(cur[le + t.jflat[q]]));
            else
                Num::mac(w, jump_cplx<Num, RT>(t, q, i, j, d, vL, vR, uj), Num::load(cur[le + t.jflat[q]]));
        }
    };
    if (!REALJ && t.jrate) jumps(std::true_type{});
    else jumps(std::false_type{});
    return Num::done(w);
}

// Shared-memory layout of prop_kernel (all 16-byte entries in storage format):
//   buf0, buf1 [win]      stage-input windows (chunk + halo on both sides)
//   xs, as     [chunk]    base value and RK accumulator of the owned entries
//   bands      [2][nb][d] A(u_j) of the current and the next slice
//   vL, vR     [nt][d]    jump tables
//   rc         [chunk]    (row, column) of the owned entries (int2)
//   cg, ca, cb [4] each   RK coefficients in the number type (8 bytes each)
template <class Num, bool REALJ>
__global__ void __launch_bounds__(GRAPE_PROP_THREADS, 1) prop_kernel(const PropArgs p) {
    using S = typename Num::store_t;
    using V = typename Num::val;
    using R = typename Num::real_t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int d = p.d, d2 = d * d;
    const int nbd = p.tab.nb * d;
    S *buf0 = reinterpret_cast<S *>(smem_raw);
    S *buf1 = buf0 + p.win;
    S *xs = buf1 + p.win;
    S *as = xs + p.chunk;
    S *bands = as + p.chunk;                 // [2][nb][d]
    S *vL = bands + 2 * nbd;                 // [nt][d]
    S *vR = vL + p.tab.nt * d;               // [nt][d]
    int2 *rc = reinterpret_cast<int2 *>(vR + p.tab.nt * d);
    R *cg = reinterpret_cast<R *>(rc + p.chunk);   // RK coefficients g, a, b
    R *ca = cg + 4;
    R *cb = cg + 8;
    const S *x_in = static_cast<const S *>(p.x_in);
    S *x_out = static_cast<S *>(p.x_out);
    S *stage_store = static_cast<S *>(p.stage_store);
    S *bound_store = static_cast<S *>(p.bound_store);

    const int rank = blockIdx.x % p.ncl;
    const int state = blockIdx.x / p.ncl;
    const int e0 = rank * p.chunk;
    const int e1 = min(e0 + p.chunk, d2);
    const int wbase = e0 - p.halo;
    const size_t soff = (size_t)state * d2;
    const int nth = blockDim.x;

    const V vzero = Num::zero();
    for (int i = threadIdx.x; i < 2 * p.win; i += nth) buf0[i] = Num::store(vzero);
    for (int i = threadIdx.x; i < p.tab.nt * d; i += nth) {
        vL[i] = Num::store(Num::from_double2(__ldg(&p.tab.vL[i])));
        vR[i] = Num::store(Num::from_double2(__ldg(&p.tab.vR[i])));
    }
    for (int e = e0 + threadIdx.x; e < e1; e += nth) rc[e - e0] = make_int2(e / d, e % d);
    if (threadIdx.x < 4) {
        cg[threadIdx.x] = Num::real_const(p.g[threadIdx.x]);
        ca[threadIdx.x] = Num::real_const(p.a[threadIdx.x]);
        cb[threadIdx.x] = Num::real_const(p.b[threadIdx.x]);
    }
    const long long nsub = p.sub_end - p.sub_begin;
    long long n_first = p.reverse ? p.sub_end - 1 : p.sub_begin;
    if (nsub <= 0) n_first = p.sub_begin;
    int jcur = (int)(n_first / p.n_rk);
    build_bands<Num>(bands, p, jcur);
    cluster_sync_all();   // every CTA of the cluster runs and has zeroed its windows

    for (int e = e0 + threadIdx.x; e < e1; e += nth) {
        const V x = Num::load(x_in[soff + e]);
        xs[e - e0] = Num::store(x);
        push_value(buf0, p, rank, e, Num::store(Num::scale(cg[0], x)));
    }
    cluster_sync_all();

    int tb = 0;
    for (long long it = 0; it < nsub; ++it) {
        const long long n = p.reverse ? p.sub_end - 1 - it : p.sub_begin + it;
        const long long tidx = p.reverse ? n + 1 : n;
        if (bound_store && ((tidx - p.sub_begin) % p.bound_step) == 0) {
            S *dst = bound_store + ((size_t)((tidx - p.sub_begin) / p.bound_step) * p.n_states) * d2 + soff;
            for (int e = e0 + threadIdx.x; e < e1; e += nth) dst[e] = xs[e - e0];
        }
        const S *A = bands + tb * nbd;
        bool flip = false;
#pragma unroll 1
        for (int s = 0; s < 4; ++s) {
            const S *cur = (s & 1) ? buf1 : buf0;
            S *nxt = (s & 1) ? buf0 : buf1;
            S *st = nullptr;                     // packed stage storage of this state
            if (stage_store)
                st = stage_store + ((size_t)((n - p.sub_begin) * 4 + p.store_map[s]) * p.n_states + state) *
                                       (size_t)(d * (d + 1) / 2);
            const R as_ = ca[s];
#pragma unroll 1
            for (int e = e0 + threadIdx.x; e < e1; e += nth) {
                const int le = e - wbase, li = e - e0;
                const int2 ij = rc[li];
                const V w = lindblad_at<Num, REALJ>(cur, le, ij.x, ij.y, d, p.tab, A, vL, vR,
                                                    p.u + (size_t)jcur * p.R);
                if (st && ij.y >= ij.x) st[ij.x * d - ij.x * (ij.x - 1) / 2 + (ij.y - ij.x)] = cur[le];
                const V x = Num::load(xs[li]);
                const V acc = Num::axpy(as_, w, s == 0 ? x : Num::load(as[li]));
                V z;
                if (s < 3) {
                    as[li] = Num::store(acc);
                    z = Num::lin2(cg[s + 1], x, cb[s + 1], w);
                } else {
                    const V nx = with_source<Num>(p, n, ij.x, ij.y, acc);
                    xs[li] = Num::store(nx);
                    z = Num::scale(cg[0], nx);
                }
                push_value(nxt, p, rank, e, Num::store(z));
            }
            if (s == 3 && it + 1 < nsub) {
                const long long nn = p.reverse ? n - 1 : n + 1;
                const int jn = (int)(nn / p.n_rk);
                if (jn != jcur) {
                    build_bands<Num>(bands + (tb ^ 1) * nbd, p, jn);
                    jcur = jn;
                    flip = true;
                }
            }
            cluster_sync_all();
        }
        if (flip) tb ^= 1;
    }
    const long long tend = p.reverse ? p.sub_begin : p.sub_end;
    if (bound_store && ((tend - p.sub_begin) % p.bound_step) == 0) {
        S *dst = bound_store + ((size_t)((tend - p.sub_begin) / p.bound_step) * p.n_states) * d2 + soff;
        for (int e = e0 + threadIdx.x; e < e1; e += nth) dst[e] = xs[e - e0];
    }
    for (int e = e0 + threadIdx.x; e < e1; e += nth) x_out[soff + e] = xs[e - e0];
}

// ---------------------------------------------------------------------------
// Hermitian propagation: every stage value is Hermitian (rho, sigma and the
// stage combinations are, and both Lindbladians preserve it), so only the
// upper triangle j >= i is computed.  CTA k of the cluster owns the upper
// entries [u0, u1) in row-major order (equal counts), and its window holds
// rows [wr0, wr0 + nrows) stored as columns [cs(r), d) with
// cs(r) = max(0, r - hb): the upper part plus the hb entries left of the
// diagonal, which are the only lower entries the stencil reads; those are
// filled with conjugate mirrors of the upper entries near the diagonal.
// Stage, boundary and output stores to HBM write full matrices (the lower
// triangle as conjugates), so every other kernel sees ordinary d x d data.
struct HWin {
    const int *tab;    // shared-memory copy of htab
    int ncl, d, hb;
};

__device__ __forceinline__ int cs_of(int r, int hb) { return r > hb ? r - hb : 0; }

// window offset of (r, c) in CTA k's window
__device__ __forceinline__ int hwin_addr(const HWin &h, int k, int r, int c) {
    const int wr0 = h.tab[GRAPE_HTAB_CTA(k) + 2];
    const int *ofs = h.tab + h.tab[GRAPE_HTAB_LISTS(h.ncl) + k];
    return ofs[r - wr0] + (c - cs_of(r, h.hb));
}

// write z at (r, c) into every window of the cluster that holds row r
template <class S>
__device__ __forceinline__ void hpush(S *buf, const HWin &h, int rank, int r, int c, S z) {
    const int *kf = h.tab + (h.tab[GRAPE_HTAB_LISTS(h.ncl) + h.ncl]);
    const int kfirst = kf[r], klast = kf[h.d + r];
    for (int k = kfirst; k <= klast; ++k) {
        S *dst = &buf[hwin_addr(h, k, r, c)];
        if (k == rank) *dst = z;
        else st_remote(map_to_rank(smem_u32(dst), (uint32_t)k), z);
    }
}

template <class Num>
__device__ __forceinline__ typename Num::store_t conj_store(typename Num::val v) {
    return Num::store(Num::conj(v));
}

__device__ __forceinline__ void st_cluster_addr(uint32_t addr, double2 v) { st_remote(addr, v); }
__device__ __forceinline__ void st_cluster_addr(uint32_t addr, float4 v) { st_remote(addr, v); }

// W = Op(z) at an owned upper entry (i, j) from its precomputed neighbour
// window addresses nb_ad: [2 b] = (i + o_b, j), [2 b + 1] = (i, j + o_b),
// [2 nb + q] = (i + oL_q, j + oR_q); -1 where the neighbour lies outside the
// matrix (its coefficient is zero there).
// D_ij = -i (A_0[i] - conj(A_0[j])) + sum over jump terms with both offsets
// 0 of vL_t[i] conj(vR_t[j]): the coefficient of X_ij itself in W_ij
template <class Num, bool REALJ>
__device__ __forceinline__ typename Num::val diag_coef(int i, int j, int d, const PropTables &t,
                                                       const typename Num::store_t *A,
                                                       const typename Num::store_t *vL,
                                                       const typename Num::store_t *vR,
                                                       const double *uj) {
    typename Num::val c = Num::zero();
    if (t.b0 >= 0) c = Num::minus_i(Num::sub_conj(Num::load(A[t.b0 * d + i]), Num::load(A[t.b0 * d + j])));
    auto jumps = [&](auto rate) {
        constexpr bool RT = decltype(rate)::value;
        for (int q = 0; q < t.nt; ++q) {
            if (!((t.jdiag >> q) & 1)) continue;
            if (REALJ) c = Num::add_real(c, jump_real<Num, RT>(t, q, i, j, d, vL, vR, uj));
            else c = Num::add(c, jump_cplx<Num, RT>(t, q, i, j, d, vL, vR, uj));
        }
    };
    if (!REALJ && t.jrate) jumps(std::true_type{});
    else jumps(std::false_type{});
    return c;
}

// Band and jump layout known at compile time (NB bands including the
// offset-0 band, which is last; the first NBR are real; NT jump terms), so
// the per-entry loops unroll and the neighbour indices can live in
// registers; ShapeAny reads the counts from the tables at run time.  The
// host picks a shape only when both directions' tables match it.
template <int NB_, int NBR_, int NT_>
struct Shape {
    static constexpr int NB = NB_, NBR = NBR_, NT = NT_;
};
using ShapeAny = Shape<0, 0, 0>;
using ShapeT = Shape<5, 2, 3>;   // transmon x resonator: bands 0, +-1 (real drive), +-Q; jumps a, b, b^dag b
using ShapeR = Shape<3, 0, 1>;   // resonator drives only: bands 0, +-Q; jump a
template <class SH> __device__ __forceinline__ int sh_nb(const PropTables &t) { return SH::NB ? SH::NB : t.nb; }
template <class SH> __device__ __forceinline__ int sh_nt(const PropTables &t) { return SH::NB ? SH::NT : t.nt; }

// The Hamiltonian bands: the first t.nbr are real for every control value
// (real multiply-adds: the same bits as the complex ones with a zero
// imaginary part, half the work), the offset-0 band is last and excluded
// (it is part of the own-entry coefficient).  x1(b), x2(b): the neighbours
// (i + o_b, j) and (i, j + o_b).  The A X terms and the X A^+ terms go to
// two accumulators (two independent dependency chains), added at the end
// (four, real and complex bands apart, measured 3 % slower).
template <class Num, class SH, class X1, class X2>
__device__ __forceinline__ typename Num::acc band_terms(const PropTables &t, const typename Num::store_t *A,
                                                        int i, int j, int d, X1 &&x1, X2 &&x2) {
    typename Num::acc wa = Num::acc_zero(), wb = Num::acc_zero();
    if constexpr (SH::NB > 0) {
#pragma unroll
        for (int b = 0; b < SH::NBR; ++b) {
            Num::mac_real(wa, Num::load_re(A[b * d + i]), x1(b));
            Num::mac_real(wb, Num::neg_real(Num::load_re(A[b * d + j])), x2(b));
        }
#pragma unroll
        for (int b = SH::NBR; b < SH::NB - 1; ++b) {
            Num::mac(wa, Num::load(A[b * d + i]), x1(b));
            Num::mac_conj_neg(wb, Num::load(A[b * d + j]), x2(b));
        }
    } else {
        const int nbo = (t.b0 >= 0) ? t.nb - 1 : t.nb;
#pragma unroll 1
        for (int b = 0; b < t.nbr; ++b) {
            Num::mac_real(wa, Num::load_re(A[b * d + i]), x1(b));
            Num::mac_real(wb, Num::neg_real(Num::load_re(A[b * d + j])), x2(b));
        }
#pragma unroll 2
        for (int b = t.nbr; b < nbo; ++b) {
            Num::mac(wa, Num::load(A[b * d + i]), x1(b));
            Num::mac_conj_neg(wb, Num::load(A[b * d + j]), x2(b));
        }
    }
    return Num::acc_add(wa, wb);
}

// jc: null, or the entry's cached coefficients of the jump terms with an
// offset (real tables only), jc[q' * jstride] for the q'-th such term
template <class Num, bool REALJ, class SH, bool JQ = false>
__device__ __forceinline__ typename Num::val lindblad_h_at(const typename Num::store_t *cur,
                                                           const short *nb_ad, int i, int j, int d,
                                                           const PropTables &t,
                                                           const typename Num::store_t *A,
                                                           const typename Num::store_t *vL,
                                                           const typename Num::store_t *vR,
                                                           const typename Num::val dij,
                                                           const double *uj,
                                                           const typename Num::real_t *jc, int jstride) {
    // neighbours outside the matrix point at the window's zero slot, so
    // every term is accumulated without a branch (adding 0 changes no bit).
    // The terms on the entry itself - the offset-0 band and the jump terms
    // with both offsets 0 - come as one coefficient D_ij (diag_coef).
    const int nb = sh_nb<SH>(t), nt = sh_nt<SH>(t);
    typename Num::acc w = band_terms<Num, SH>(t, A, i, j, d, [&](int b) { return Num::load(cur[nb_ad[2 * b]]); },
                                              [&](int b) { return Num::load(cur[nb_ad[2 * b + 1]]); });
    w = Num::acc_minus_i(w);
    Num::mac(w, dij, Num::load(cur[nb_ad[2 * nb + nt]]));
    if (REALJ && jc) {
        int qq = 0;
        auto term = [&](int q) {
            if ((t.jdiag >> q) & 1) return;
            // JQ: coefficient q of a per-term array (registers); else the
            // qq-th term with an offset in the per-entry cache
            Num::mac_real(w, jc[(JQ ? q : qq) * jstride], Num::load(cur[nb_ad[2 * nb + q]]));
            ++qq;
        };
        if constexpr (SH::NB > 0) {
#pragma unroll
            for (int q = 0; q < SH::NT; ++q) term(q);
        } else {
#pragma unroll 1
            for (int q = 0; q < nt; ++q) term(q);
        }
        return Num::raw(w);
    }
    auto jumps = [&](auto rate) {
        constexpr bool RT = decltype(rate)::value;
        auto term = [&](int q) {
            if ((t.jdiag >> q) & 1) return;
            const int aJ = nb_ad[2 * nb + q];
            if (REALJ) Num::mac_real(w, jump_real<Num, RT>(t, q, i, j, d, vL, vR, uj), Num::load(cur[aJ]));
            else Num::mac(w, jump_cplx<Num, RT>(t, q, i, j, d, vL, vR, uj), Num::load(cur[aJ]));
        };
        if constexpr (SH::NB > 0) {
#pragma unroll
            for (int q = 0; q < SH::NT; ++q) term(q);
        } else {
#pragma unroll 1
            for (int q = 0; q < nt; ++q) term(q);
        }
    };
    if (!REALJ && t.jrate) jumps(std::true_type{});
    else jumps(std::false_type{});
    return Num::raw(w);
}

// full-matrix store of upper entry (i, j) and its conjugate mirror
template <class Num>
__device__ __forceinline__ void store_herm(typename Num::store_t *dst, int d, int i, int j,
                                           typename Num::store_t v) {
    dst[(size_t)i * d + j] = v;
    if (j != i) dst[(size_t)j * d + i] = conj_store<Num>(Num::load(v));
}

// push value v of entry (r, c) to every window holding row r: rowtab holds,
// per row, the target count and each target's distributed-shared-memory
// address of (r, 0) in buf0 (buffer offset boff selects buf1)
template <class S>
__device__ __forceinline__ void hpush_pre(const uint32_t *rowtab, int rstride, int rrow, int c,
                                          uint32_t boff, S v) {
    const uint32_t *e = rowtab + rrow * rstride;
    const int n = (int)e[0];
    for (int t = 1; t <= n; ++t) st_cluster_addr(e[t] + boff + (uint32_t)c * (uint32_t)sizeof(S), v);
}

// Distributed-shared-memory pushes with transaction counting: st.async
// writes 16 bytes into a peer CTA's window and counts them on the peer's
// mbarrier of that window (complete_tx), so the writer never waits for the
// store to complete; the reader waits on its own mbarrier until every byte
// its window expects in the phase has arrived.  Pushes into the CTA's own
// window are ordinary shared-memory stores, published by every thread's
// arrival (release) on the same mbarrier.
__device__ __forceinline__ void st_async16(uint32_t addr, float4 v, uint32_t mbar) {
    asm volatile("st.async.weak.shared::cluster.mbarrier::complete_tx::bytes.v4.b32 [%0], {%1, %2, %3, %4}, [%5];"
                 ::"r"(addr), "r"(__float_as_uint(v.x)), "r"(__float_as_uint(v.y)), "r"(__float_as_uint(v.z)),
                 "r"(__float_as_uint(v.w)), "r"(mbar)
                 : "memory");
}
__device__ __forceinline__ void st_async16(uint32_t addr, double2 v, uint32_t mbar) {
    asm volatile("st.async.weak.shared::cluster.mbarrier::complete_tx::bytes.v2.b64 [%0], {%1, %2}, [%3];"
                 ::"r"(addr), "l"(__double_as_longlong(v.x)), "l"(__double_as_longlong(v.y)), "r"(mbar)
                 : "memory");
}
__device__ __forceinline__ void st_local16(uint32_t addr, float4 v) {
    asm volatile("st.shared.v4.f32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "f"(v.x), "f"(v.y), "f"(v.z), "f"(v.w)
                 : "memory");
}
__device__ __forceinline__ void st_local16(uint32_t addr, double2 v) {
    asm volatile("st.shared.v2.f64 [%0], {%1, %2};" ::"r"(addr), "d"(v.x), "d"(v.y) : "memory");
}
__device__ __forceinline__ void mbar_init(uint32_t mbar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(mbar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// the one arrival of a phase, announcing the bytes the phase expects
__device__ __forceinline__ void mbar_expect(uint32_t mbar, uint32_t bytes) {
    asm volatile("{\n\t.reg .b64 st;\n\t"
                 "mbarrier.arrive.expect_tx.release.cta.shared::cta.b64 st, [%0], %1;\n\t}" ::"r"(mbar),
                 "r"(bytes)
                 : "memory");
}
// a plain arrival (release: the arriving thread's earlier shared-memory
// stores are visible to a thread whose wait on the phase succeeds)
__device__ __forceinline__ void mbar_arrive(uint32_t mbar) {
    asm volatile("{\n\t.reg .b64 st;\n\t"
                 "mbarrier.arrive.release.cta.shared::cta.b64 st, [%0];\n\t}" ::"r"(mbar)
                 : "memory");
}
// bounded wait for the phase of the given parity: false when it gave up
// after `cycles` SM clock cycles (about a second for 2^31)
__device__ __forceinline__ bool mbar_wait(uint32_t mbar, uint32_t parity, long long cycles) {
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(mbar), "r"(parity)
                     : "memory");
        if (done) return true;
        if (clock64() - t0 > cycles) return false;
    }
}
// bulk asynchronous copy (TMA engine) of `bytes` from global memory into the
// CTA's shared memory, counted on its mbarrier; both addresses and the size
// are multiples of 16 bytes
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void *src, uint32_t bytes, uint32_t mbar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(mbar)
                 : "memory");
}
// the two halves of the cluster barrier without memory ordering: they only
// keep a CTA from overwriting a window a peer may still be reading
__device__ __forceinline__ void cluster_arrive_relaxed() {
    __syncwarp();
    asm volatile("barrier.cluster.arrive.relaxed;" ::: "memory");
}
__device__ __forceinline__ void cluster_wait_only() {
    asm volatile("barrier.cluster.wait;" ::: "memory");
}

// push value v of entry (r, c) to every window holding row r: rowtab holds,
// per row, the target count and per target the address of (r, 0) in buf0
// (shared::cluster for a peer, shared::cta for the own CTA) and the peer's
// mbarrier of buf0 (0 for the own CTA); boff selects the next window and
// moff its mbarrier
template <class S>
__device__ __forceinline__ void hpush_async(const uint32_t *rowtab, int rstride, int rrow, int c, uint32_t boff,
                                            uint32_t moff, S v) {
    const uint32_t *e = rowtab + rrow * rstride;
    const int n = (int)e[0];
    for (int t = 0; t < n; ++t) {
        const uint32_t a = e[1 + 2 * t] + boff + (uint32_t)c * (uint32_t)sizeof(S);
        const uint32_t m = e[2 + 2 * t];
        if (m) st_async16(a, v, m + moff);
        else st_local16(a, v);
    }
}

// Shared memory: two mbarriers (16 B); buf0, buf1 [maxwin + 1] (the last
// entry of each stays zero); xs, as [cu]; D [cu] when p.fold; z [cu] when
// p.defer; bands
// [2][nb][d]; vL, vR [nt][d]; rc [cu] (int2); 12 RK coefficients; jump
// coefficients [njt][cu] (real_t) when p.jcache; htab copy (ints); row push
// table [rt_rows][2 ncl + 1] (u32); neighbour addresses [cu][ns + 1] (i16).
//
// Stage g reads window g mod 2 and pushes the next stage's input into
// window (g + 1) mod 2.  Synchronisation per stage (cluster of ncl > 1):
//  - wait on the window's mbarrier: every byte that peers push into it for
//    this stage has landed (one thread announced the count when the phase
//    began, 16 B per window slot a peer owns) and every thread of the CTA
//    arrived after its own pushes into it (a phase needs 1 + blockDim.x
//    arrivals), so no CTA barrier separates the stages;
//  - wait on the cluster barrier that every thread arrived at after
//    computing the previous stage: no peer still reads the window the
//    pushes below overwrite;
//  - compute the owned entries and push each as it is computed;
//  - arrive on the next window's mbarrier, arrive at the cluster barrier
//    (relaxed: it orders nothing); a CTA barrier follows only the per-slice
//    rebuild of the band table.
// With p.defer (tiles with several entries per thread) the next values wait
// in the z row and the cluster wait comes after the compute, just before
// the pushes (the same values; measured slower, off by default).
// No release fence waits for the pushes or the stage stores.  Every
// mbarrier wait is bounded: when one gives up, the error word gbar[2] is set
// to 2, later waits are skipped and the results are invalid (the host
// reports GRAPE_ETIMEOUT).  A one-CTA cluster pushes only into itself and
// needs only the CTA barrier.
// SH: the band and jump layout (ShapeAny: from the tables); ONE: every
// thread owns at most one upper entry (cu <= threads), so the entry's
// neighbour indices stay in registers for the whole launch.
template <class Num, bool REALJ, class SH, bool ONE>
__global__ void __launch_bounds__(GRAPE_PROP_THREADS, 1) prop_h_kernel(const PropArgs p) {
    using S = typename Num::store_t;
    using V = typename Num::val;
    using R = typename Num::real_t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_count, s_err;
    const int d = p.d, d2 = d * d;
    const int NU = d * (d + 1) / 2;
    const int nbd = p.tab.nb * d;
    const int wst = p.maxwin + 1;                // window stride; slot maxwin is the zero slot
    uint64_t *mbar = reinterpret_cast<uint64_t *>(smem_raw);
    S *buf0 = reinterpret_cast<S *>(smem_raw + 16);
    S *buf1 = buf0 + wst;
    S *xs = buf1 + wst;
    S *as = xs + p.cu;
    S *Dt = as + p.cu;                           // [cu] own-entry coefficients when p.fold
    S *zr = Dt + (p.fold ? p.cu : 0);            // [cu] next stage values when p.defer
    S *bands = zr + (p.defer ? p.cu : 0);
    S *vL = bands + 2 * nbd;
    S *vR = vL + p.tab.nt * d;
    int2 *rc = reinterpret_cast<int2 *>(vR + p.tab.nt * d);
    R *cg = reinterpret_cast<R *>(rc + p.cu);
    R *ca = cg + 4;
    R *cb = cg + 8;
    const int njt = p.tab.nt - __popc(p.tab.jdiag);   // jump terms with an offset
    const bool jcache = REALJ && p.jcache;
    R *jc = cg + 12;                             // [njt][cu] when jcache
    int *tab = reinterpret_cast<int *>(jc + (jcache ? njt * p.cu : 0));
    const int rstride = 2 * p.ncl + 1;
    uint32_t *rowtab = reinterpret_cast<uint32_t *>(tab + p.htab_len);
    short *nbad = reinterpret_cast<short *>(rowtab + p.rt_rows * rstride);
    const int ns = SH::NB ? 2 * SH::NB + SH::NT : 2 * p.tab.nb + p.tab.nt;   // neighbour slots; slot ns = own address
    const int nstride = ns + 1;
    const S *x_in = static_cast<const S *>(p.x_in);
    S *x_out = static_cast<S *>(p.x_out);
    S *stage_store = static_cast<S *>(p.stage_store);
    S *bound_store = static_cast<S *>(p.bound_store);
    const int rank = blockIdx.x % p.ncl;
    const int state = blockIdx.x / p.ncl;
    const size_t soff = (size_t)state * d2;
    const int nth = blockDim.x;
    const int hb = p.hb;
    const bool clu = p.ncl > 1;
    const uint32_t mbar_sa = smem_u32(mbar);

    if (threadIdx.x == 0) {
        s_count = 0;
        s_err = 0;
        // per phase: the announcing arrival (expect_tx) and one arrival of
        // every thread after its pushes into the window
        mbar_init(mbar_sa, 1u + (uint32_t)blockDim.x);
        mbar_init(mbar_sa + 8, 1u + (uint32_t)blockDim.x);
        mbar_init_fence();
    }
    for (int i = threadIdx.x; i < p.htab_len; i += nth) tab[i] = __ldg(&p.htab[i]);
    const V vzero = Num::zero();
    for (int i = threadIdx.x; i < 2 * wst; i += nth) buf0[i] = Num::store(vzero);
    for (int i = threadIdx.x; i < p.tab.nt * d; i += nth) {
        vL[i] = Num::store(Num::from_double2(__ldg(&p.tab.vL[i])));
        vR[i] = Num::store(Num::from_double2(__ldg(&p.tab.vR[i])));
    }
    if (threadIdx.x < 4) {
        cg[threadIdx.x] = Num::real_const(p.g[threadIdx.x]);
        ca[threadIdx.x] = Num::real_const(p.a[threadIdx.x]);
        cb[threadIdx.x] = Num::real_const(p.b[threadIdx.x]);
    }
    const long long nsub = p.sub_end - p.sub_begin;
    long long n_first = p.reverse ? p.sub_end - 1 : p.sub_begin;
    if (nsub <= 0) n_first = p.sub_begin;
    int jcur = (int)(n_first / p.n_rk);
    build_bands<Num>(bands, p, jcur);
    __syncthreads();
    const int u0 = tab[GRAPE_HTAB_CTA(rank) + 0], u1 = tab[GRAPE_HTAB_CTA(rank) + 1];
    const int wr0 = tab[GRAPE_HTAB_CTA(rank) + 2], nrows = tab[GRAPE_HTAB_CTA(rank) + 3];
    const int *ofs = tab + tab[GRAPE_HTAB_LISTS(p.ncl) + rank];
    const int *kfl = tab + tab[GRAPE_HTAB_LISTS(p.ncl) + p.ncl];   // kfirst[d], klast[d]
    // (row, column) of the owned upper entries (row-major offset of row i is
    // i d - i (i - 1) / 2), their neighbours' window addresses and, for real
    // jump tables, their jump coefficients (fixed for the whole sweep)
    for (int u = u0 + threadIdx.x; u < u1; u += nth) {
        const double b2 = 2.0 * d + 1.0;
        int i = (int)floor(0.5 * (b2 - sqrt(b2 * b2 - 8.0 * (double)u)));
        i = max(0, min(d - 1, i));
        while (i > 0 && (long long)i * d - (long long)i * (i - 1) / 2 > u) --i;
        while (i + 1 < d && (long long)(i + 1) * d - (long long)(i + 1) * i / 2 <= u) ++i;
        const int j = i + (int)(u - ((long long)i * d - (long long)i * (i - 1) / 2));
        rc[u - u0] = make_int2(i, j);
        short *na = nbad + (size_t)(u - u0) * nstride;
        const int own = ofs[i - wr0] + (j - cs_of(i, hb));
        na[ns] = (short)own;
        const short zs = (short)p.maxwin;
        for (int b = 0; b < p.tab.nb; ++b) {
            const int o = p.tab.off[b], r = i + o, c = j + o;
            na[2 * b] = (r >= 0 && r < d) ? (short)(ofs[r - wr0] + (j - cs_of(r, hb))) : zs;
            na[2 * b + 1] = (c >= 0 && c < d) ? (short)(own + o) : zs;
        }
        for (int q = 0; q < p.tab.nt; ++q) {
            const int r = i + p.tab.joL[q], c = j + p.tab.joR[q];
            na[2 * p.tab.nb + q] =
                (r >= 0 && r < d && c >= 0 && c < d) ? (short)(ofs[r - wr0] + (c - cs_of(r, hb))) : zs;
        }
        if (jcache) {
            int qq = 0;
            for (int q = 0; q < p.tab.nt; ++q) {
                if ((p.tab.jdiag >> q) & 1) continue;
                jc[qq * p.cu + (u - u0)] = jump_real<Num, false>(p.tab, q, i, j, d, vL, vR, nullptr);
                ++qq;
            }
        }
    }
    // window slots written by peers each stage (16 B each): slot (r, c) of
    // the window holds the upper entry (r, c), c >= r, or the mirror of
    // (c, r); its writer is the owner of that upper entry
    if (clu) {
        const int cu = p.cu;
        int cnt = 0;
        for (int lr = threadIdx.x; lr < nrows; lr += nth) {
            const int r = wr0 + lr;
            for (int c = cs_of(r, hb); c < d; ++c) {
                const int ur = c >= r ? r * d - r * (r - 1) / 2 + (c - r) : c * d - c * (c - 1) / 2 + (r - c);
                if (ur / cu != rank) ++cnt;
            }
        }
        if (cnt) atomicAdd(&s_count, cnt);
    }
    // push targets of the rows this CTA writes: its own rows and, for the
    // mirrors, up to hb rows below
    int rfirst = 0, rlast = -1;
    if (u1 > u0) {
        // rows of the first and last owned entries (same formula as above)
        auto row_of = [&](int u) {
            const double b2 = 2.0 * d + 1.0;
            int i = (int)floor(0.5 * (b2 - sqrt(b2 * b2 - 8.0 * (double)u)));
            i = max(0, min(d - 1, i));
            while (i > 0 && (long long)i * d - (long long)i * (i - 1) / 2 > u) --i;
            while (i + 1 < d && (long long)(i + 1) * d - (long long)(i + 1) * i / 2 <= u) ++i;
            return i;
        };
        rfirst = row_of(u0);
        rlast = min(d - 1, row_of(u1 - 1) + hb);
    }
    const uint32_t buf0_sa = smem_u32(buf0);
    for (int r = rfirst + threadIdx.x; r <= rlast; r += nth) {
        uint32_t *e = rowtab + (r - rfirst) * rstride;
        const int kf = kfl[r], kl = kfl[d + r];
        int n = 0;
        for (int k = kf; k <= kl; ++k) {
            const int wk = tab[GRAPE_HTAB_CTA(k) + 2];
            const int *ofk = tab + tab[GRAPE_HTAB_LISTS(p.ncl) + k];
            const int base = ofk[r - wk] - cs_of(r, hb);       // entry index of (r, 0), may be < 0
            const uint32_t boffs = (uint32_t)(base * (int)sizeof(S));
            if (k == rank) {
                e[1 + 2 * n] = buf0_sa + boffs;
                e[2 + 2 * n] = 0u;
            } else {
                e[1 + 2 * n] = map_to_rank(buf0_sa, (uint32_t)k) + boffs;
                e[2 + 2 * n] = map_to_rank(mbar_sa, (uint32_t)k);
            }
            ++n;
        }
        e[0] = (uint32_t)n;
    }
    cluster_sync_all();   // every CTA runs, windows zeroed, mbarriers initialised, tables built
    const uint32_t expect = (uint32_t)s_count * (uint32_t)sizeof(S);
    const long long limit = 1LL << 31;          // SM cycles a window wait may take
    const uint32_t boff1 = (uint32_t)(wst * (int)sizeof(S));

    // the initial stage input (window 0)
    if (clu && threadIdx.x == 0) mbar_expect(mbar_sa, expect);
    for (int u = u0 + threadIdx.x; u < u1; u += nth) {
        const int2 ij = rc[u - u0];
        const V x = Num::load(x_in[soff + (size_t)ij.x * d + ij.y]);
        xs[u - u0] = Num::store(x);
        const V z = Num::scale(cg[0], x);
        hpush_async(rowtab, rstride, ij.x - rfirst, ij.y, 0u, 0u, Num::store(z));
        if (ij.y > ij.x && ij.y - ij.x <= hb)
            hpush_async(rowtab, rstride, ij.y - rfirst, ij.x, 0u, 0u, conj_store<Num>(z));
    }
    if (clu) {
        mbar_arrive(mbar_sa);
        cluster_arrive_relaxed();
    }
    __syncthreads();

    const bool unit_g = (p.g[1] == 1.0 && p.g[2] == 1.0 && p.g[3] == 1.0);   // forward RK4
    constexpr int NSC = SH::NB ? 2 * SH::NB + SH::NT + 1 : 1;
    constexpr int NJQ = SH::NB ? SH::NT : 1;
    // ONE: the entry's neighbour indices, row and column, base value, RK
    // accumulator, own-entry coefficient and jump coefficients in registers
    short nreg[NSC];
    int2 ijr = make_int2(0, 0);
    V xr = Num::zero(), ar = Num::zero(), dr = Num::zero();
    R jreg[NJQ];
#pragma unroll
    for (int q = 0; q < NJQ; ++q) jreg[q] = Num::real_const(0.0);
    if constexpr (ONE) {
        const bool mine = u0 + (int)threadIdx.x < u1;
        const short *na0 = nbad + (size_t)threadIdx.x * nstride;
#pragma unroll
        for (int k = 0; k < NSC; ++k) nreg[k] = mine ? na0[k] : (short)0;
        if (mine) {
            ijr = rc[threadIdx.x];
            xr = Num::load(xs[threadIdx.x]);
            if (jcache) {
                int qq = 0;
#pragma unroll
                for (int q = 0; q < NJQ; ++q) {
                    if ((p.tab.jdiag >> q) & 1) continue;
                    jreg[q] = jc[qq * p.cu + threadIdx.x];
                    ++qq;
                }
            }
        }
    }
    int tb = 0;
    uint32_t g = 0;                              // stages done in this launch
    bool dfresh = true;                          // D table to (re)build for this slice
    for (long long it = 0; it < nsub; ++it) {
        const long long n = p.reverse ? p.sub_end - 1 - it : p.sub_begin + it;
        const long long tidx = p.reverse ? n + 1 : n;
        if (bound_store && ((tidx - p.sub_begin) % p.bound_step) == 0) {
            S *dst = bound_store + ((size_t)((tidx - p.sub_begin) / p.bound_step) * p.n_states) * d2 + soff;
            for (int u = u0 + threadIdx.x; u < u1; u += nth)
                store_herm<Num>(dst, d, rc[u - u0].x, rc[u - u0].y, xs[u - u0]);
        }
        const S *A = bands + tb * nbd;
        const double *uj = p.u + (size_t)jcur * p.R;   // controls of the current slice
        bool flip = false;
#pragma unroll 1
        for (int s = 0; s < 4; ++s) {
            const S *cur = (s & 1) ? buf1 : buf0;
            const uint32_t boff = (s & 1) ? 0u : boff1;          // next window
            const uint32_t moff = (s & 1) ? 0u : 8u;             // its mbarrier
            if (clu) {
                if (!s_err && !mbar_wait(mbar_sa + (g & 1) * 8, (g >> 1) & 1, limit)) {
                    s_err = 1;
                    atomicExch(&p.gbar[2], 2u);
                }
                if (threadIdx.x == 0 && !s_err) mbar_expect(mbar_sa + moff, expect);
            }
            S *st = nullptr;                     // packed stage storage of this state
            if (stage_store)
                st = stage_store + ((size_t)((n - p.sub_begin) * 4 + p.store_map[s]) * p.n_states + state) * NU;
            const R as_ = ca[s];
            if (clu && !p.defer) cluster_wait_only();
#pragma unroll 1
            for (int u = u0 + threadIdx.x; u < u1; u += nth) {
                const int li = u - u0;
                const int2 ij = ONE ? ijr : rc[li];
                const short *na;
                if constexpr (ONE) na = nreg;
                else na = nbad + (size_t)li * nstride;
                if (st) st[u] = cur[na[ns]];     // the stage input itself, packed
                // own-entry coefficient: cached per slice (the entry is thread-private,
                // so no barrier is needed) or recomputed when there is no room
                V dij;
                if constexpr (ONE) {
                    if (s == 0 && dfresh) dr = diag_coef<Num, REALJ>(ij.x, ij.y, d, p.tab, A, vL, vR, uj);
                    dij = dr;
                } else if (p.fold) {
                    if (s == 0 && dfresh) Dt[li] = Num::store(diag_coef<Num, REALJ>(ij.x, ij.y, d, p.tab, A, vL, vR, uj));
                    dij = Num::load(Dt[li]);
                } else {
                    dij = diag_coef<Num, REALJ>(ij.x, ij.y, d, p.tab, A, vL, vR, uj);
                }
                V w;
                if constexpr (ONE)
                    w = lindblad_h_at<Num, REALJ, SH, true>(cur, na, ij.x, ij.y, d, p.tab, A, vL, vR, dij, uj,
                                                            jcache ? jreg : nullptr, 1);
                else
                    w = lindblad_h_at<Num, REALJ, SH>(cur, na, ij.x, ij.y, d, p.tab, A, vL, vR, dij, uj,
                                                      jcache ? jc + li : nullptr, p.cu);
                const V x = ONE ? xr : Num::load(xs[li]);
                const V acc = Num::axpy(as_, w, s == 0 ? x : (ONE ? ar : Num::load(as[li])));
                V z;
                if (s < 3) {
                    if constexpr (ONE) ar = acc;
                    else as[li] = Num::store(acc);
                    z = unit_g ? Num::axpy(cb[s + 1], w, x) : Num::lin2(cg[s + 1], x, cb[s + 1], w);
                } else {
                    const V nx = with_source<Num>(p, n, ij.x, ij.y, acc);
                    xs[li] = Num::store(nx);         // kept for the boundary and final stores
                    if constexpr (ONE) xr = nx;
                    z = Num::scale(cg[0], nx);
                }
                if (p.defer) {
                    zr[li] = Num::store(z);
                } else {
                    hpush_async(rowtab, rstride, ij.x - rfirst, ij.y, boff, moff, Num::store(z));
                    if (ij.y > ij.x && ij.y - ij.x <= hb)
                        hpush_async(rowtab, rstride, ij.y - rfirst, ij.x, boff, moff, conj_store<Num>(z));
                }
            }
            if (p.defer) {
                if (clu) cluster_wait_only();    // no peer still reads the next window
#pragma unroll 1
                for (int u = u0 + threadIdx.x; u < u1; u += nth) {
                    const int li = u - u0;
                    const int2 ij = rc[li];
                    const S z = zr[li];
                    hpush_async(rowtab, rstride, ij.x - rfirst, ij.y, boff, moff, z);
                    if (ij.y > ij.x && ij.y - ij.x <= hb)
                        hpush_async(rowtab, rstride, ij.y - rfirst, ij.x, boff, moff, conj_store<Num>(Num::load(z)));
                }
            }
            if (s == 3 && it + 1 < nsub) {
                const long long nn = p.reverse ? n - 1 : n + 1;
                const int jn = (int)(nn / p.n_rk);
                if (jn != jcur) {
                    build_bands<Num>(bands + (tb ^ 1) * nbd, p, jn);
                    __syncthreads();             // the new table before the next stage reads it
                    jcur = jn;
                    flip = true;
                }
            }
            if (clu) {
                // the own-window pushes reach the CTA's readers through the
                // window's mbarrier (every thread arrives after its pushes)
                mbar_arrive(mbar_sa + moff);
                cluster_arrive_relaxed();
            } else {
                __syncthreads();
            }
            ++g;
        }
        if (flip) tb ^= 1;
        dfresh = flip;
    }
    if (clu) {
        // the last pushes: the matching cluster wait, then every byte peers
        // pushed into this CTA has landed before it exits
        cluster_wait_only();
        if (!s_err && !mbar_wait(mbar_sa + (g & 1) * 8, (g >> 1) & 1, limit)) atomicExch(&p.gbar[2], 2u);
    }
    const long long tend = p.reverse ? p.sub_begin : p.sub_end;
    if (bound_store && ((tend - p.sub_begin) % p.bound_step) == 0) {
        S *dst = bound_store + ((size_t)((tend - p.sub_begin) / p.bound_step) * p.n_states) * d2 + soff;
        for (int u = u0 + threadIdx.x; u < u1; u += nth)
            store_herm<Num>(dst, d, rc[u - u0].x, rc[u - u0].y, xs[u - u0]);
    }
    for (int u = u0 + threadIdx.x; u < u1; u += nth)
        store_herm<Num>(x_out + soff, d, rc[u - u0].x, rc[u - u0].y, xs[u - u0]);
}

// ---------------------------------------------------------------------------
// Grid kernel for states too large for a cluster's shared memory (d = 600:
// rho is 5.76 MB): nct CTAs per state, at most one per SM, all resident (a
// cooperative launch).  The CTAs share a state's upper triangle as the
// Hermitian cluster kernel's CTAs do (contiguous entry ranges, compact row
// windows of rows first - omax .. last + omax, the same neighbour address
// tables and the same per-entry arithmetic, so the same bits), but a window
// lives in the CTA's shared memory only while one stage is computed: the
// stage values themselves live as full matrices in two global buffers
// (L2-resident), each upper entry written with its conjugate mirror.  Per
// stage a CTA
//  - waits until every neighbour CTA - one that writes a row of its window
//    or holds a row it writes - has finished the previous stage (a flag per
//    CTA counting finished push rounds, release/acquire at GPU scope): the
//    rows it reads are complete, and no neighbour still reads the buffer it
//    is about to write;
//  - loads its window rows from the buffer (cp.async through L2 only: the
//    non-coherent L1 could hold lines of two stages ago);
//  - computes its entries from shared memory and writes them, with their
//    mirrors, to the other buffer; then raises its flag.
// Only neighbours wait for one another (no grid-wide barrier).  Every wait
// is bounded: after spin_limit polls the error word gbar[2] is set to 1 and
// later waits are skipped (results invalid, GRAPE_ETIMEOUT on the host), so
// a fault cannot hang the GPU.
__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release_gpu(unsigned *p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ void cp_async_cg16(void *smem_dst, const void *gsrc) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_u32(smem_dst)), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// Shared memory: win [maxwin + 1] (the last entry stays zero); xs, as [cu];
// D [cu] when p.fold; bands [nb][d] (one table: at a slice change it is
// rebuilt at the start of the next stage, while no thread reads it); rc
// [cu] (int2); 12 RK coefficients; jump coefficients [njt][cu] when
// p.jcache; htab copy (ints); neighbour addresses [cu][ns + 1] (i16).  The
// jump tables are read from global memory.
template <class Num, bool REALJ, class SH>
__global__ void __launch_bounds__(GRAPE_GRID_THREADS, 1) prop_g_kernel(const PropArgs p) {
    using S = typename Num::store_t;
    using V = typename Num::val;
    using R = typename Num::real_t;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_err;
    const int d = p.d;
    const size_t d2 = (size_t)d * d;
    const int NU = d * (d + 1) / 2;
    const int nbd = p.tab.nb * d;
    const int wst = p.maxwin + 1;
    S *win = reinterpret_cast<S *>(smem_raw);
    S *xs = win + wst;
    S *as = xs + p.cu;
    S *Dt = as + p.cu;
    S *bands = Dt + (p.fold ? p.cu : 0);
    const S *vL = static_cast<const S *>(p.tab.vLs);
    const S *vR = static_cast<const S *>(p.tab.vRs);
    int2 *rc = reinterpret_cast<int2 *>(bands + nbd);
    R *cg = reinterpret_cast<R *>(rc + p.cu);
    R *ca = cg + 4;
    R *cb = cg + 8;
    const int njt = p.tab.nt - __popc(p.tab.jdiag);
    const bool jcache = REALJ && p.jcache;
    R *jc = cg + 12;
    int *tab = reinterpret_cast<int *>(jc + (jcache ? njt * p.cu : 0));
    short *nbad = reinterpret_cast<short *>(tab + p.htab_len);
    const int ns = SH::NB ? 2 * SH::NB + SH::NT : 2 * p.tab.nb + p.tab.nt;
    const int nstride = ns + 1;
    const int nct = p.ncl;                       // CTAs per state
    const int rank = blockIdx.x % nct;
    const int state = blockIdx.x / nct;
    S *gb0 = static_cast<S *>(p.gbuf) + (size_t)state * d2;
    S *gb1 = static_cast<S *>(p.gbuf) + (size_t)(p.n_states + state) * d2;
    const S *x_in = static_cast<const S *>(p.x_in) + (size_t)state * d2;
    S *x_out = static_cast<S *>(p.x_out) + (size_t)state * d2;
    S *stage_store = static_cast<S *>(p.stage_store);
    S *bound_store = static_cast<S *>(p.bound_store);
    unsigned *flags = p.gflag + (size_t)state * nct;   // finished push rounds per CTA of the state
    const int *nbr = p.ntab + (size_t)rank * p.ntab_stride;   // [count, ranks...]
    const int nth = blockDim.x;
    const int hb = p.hb;

    if (threadIdx.x == 0) s_err = 0;
    for (int i = threadIdx.x; i < p.htab_len; i += nth) tab[i] = __ldg(&p.htab[i]);
    const V vzero = Num::zero();
    for (int i = threadIdx.x; i < wst; i += nth) win[i] = Num::store(vzero);
    if (threadIdx.x < 4) {
        cg[threadIdx.x] = Num::real_const(p.g[threadIdx.x]);
        ca[threadIdx.x] = Num::real_const(p.a[threadIdx.x]);
        cb[threadIdx.x] = Num::real_const(p.b[threadIdx.x]);
    }
    const long long nsub = p.sub_end - p.sub_begin;
    long long n_first = p.reverse ? p.sub_end - 1 : p.sub_begin;
    if (nsub <= 0) n_first = p.sub_begin;
    int jcur = (int)(n_first / p.n_rk);
    build_bands<Num>(bands, p, jcur);
    __syncthreads();
    const int u0 = tab[GRAPE_HTAB_CTA(rank) + 0], u1 = tab[GRAPE_HTAB_CTA(rank) + 1];
    const int wr0 = tab[GRAPE_HTAB_CTA(rank) + 2], nrows = tab[GRAPE_HTAB_CTA(rank) + 3];
    const int *ofs = tab + tab[GRAPE_HTAB_LISTS(nct) + rank];
    for (int u = u0 + threadIdx.x; u < u1; u += nth) {
        const double b2 = 2.0 * d + 1.0;
        int i = (int)floor(0.5 * (b2 - sqrt(b2 * b2 - 8.0 * (double)u)));
        i = max(0, min(d - 1, i));
        while (i > 0 && (long long)i * d - (long long)i * (i - 1) / 2 > u) --i;
        while (i + 1 < d && (long long)(i + 1) * d - (long long)(i + 1) * i / 2 <= u) ++i;
        const int j = i + (int)(u - ((long long)i * d - (long long)i * (i - 1) / 2));
        rc[u - u0] = make_int2(i, j);
        short *na = nbad + (size_t)(u - u0) * nstride;
        const int own = ofs[i - wr0] + (j - cs_of(i, hb));
        na[ns] = (short)own;
        const short zs = (short)p.maxwin;
        for (int b = 0; b < p.tab.nb; ++b) {
            const int o = p.tab.off[b], r = i + o, c = j + o;
            na[2 * b] = (r >= 0 && r < d) ? (short)(ofs[r - wr0] + (j - cs_of(r, hb))) : zs;
            na[2 * b + 1] = (c >= 0 && c < d) ? (short)(own + o) : zs;
        }
        for (int q = 0; q < p.tab.nt; ++q) {
            const int r = i + p.tab.joL[q], c = j + p.tab.joR[q];
            na[2 * p.tab.nb + q] =
                (r >= 0 && r < d && c >= 0 && c < d) ? (short)(ofs[r - wr0] + (c - cs_of(r, hb))) : zs;
        }
        if (jcache) {
            int qq = 0;
            for (int q = 0; q < p.tab.nt; ++q) {
                if ((p.tab.jdiag >> q) & 1) continue;
                jc[qq * p.cu + (u - u0)] = jump_real<Num, false>(p.tab, q, i, j, d, vL, vR, nullptr);
                ++qq;
            }
        }
    }
    // the initial stage input (push round 1, buffer 0)
    for (int u = u0 + threadIdx.x; u < u1; u += nth) {
        const int2 ij = rc[u - u0];
        const V x = Num::load(x_in[(size_t)ij.x * d + ij.y]);
        xs[u - u0] = Num::store(x);
        store_herm<Num>(gb0, d, ij.x, ij.y, Num::store(Num::scale(cg[0], x)));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        st_release_gpu(&flags[rank], 1u);
    }
    // waits until every neighbour has finished `round` push rounds (thread 0),
    // then loads the window rows from `src` (the stage's input buffer)
    const int nnb = nbr[0];
    int band_next = -1;                          // slice whose bands are rebuilt at the next stage
    auto wait_and_load = [&](unsigned round, const S *src) {
        if (p.spin_limit <= 0) {                 // a limit of zero polls gives up at once
            if (threadIdx.x == 0 && !s_err) {
                atomicExch(&p.gbar[2], 1u);
                s_err = 1;
            }
            __syncthreads();                     // s_err as thread 0 left it
        }
        if (threadIdx.x < nnb && !s_err) {       // one thread per neighbour, all at once
            const unsigned *f = &flags[nbr[1 + threadIdx.x]];
            long long it = 0;
            while (ld_acquire_gpu(f) < round) {
                if (ld_acquire_gpu(&p.gbar[2]) != 0u || ++it > p.spin_limit) {
                    atomicExch(&p.gbar[2], 1u);
                    s_err = 1;
                    break;
                }
            }
        }
        __syncthreads();
        if (band_next >= 0) {                    // no thread reads the table now
            build_bands<Num>(bands, p, band_next);
            band_next = -1;
        }
        const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = nth >> 5;
        for (int lr = warp; lr < nrows; lr += nwarps) {
            const int r = wr0 + lr;
            const int c0 = cs_of(r, hb), n = d - c0;
            S *dst = win + ofs[lr];
            const S *srow = src + (size_t)r * d + c0;
            for (int c = lane; c < n; c += 32) cp_async_cg16(dst + c, srow + c);
        }
        cp_async_wait_all();
        __syncthreads();
    };

    const bool unit_g = (p.g[1] == 1.0 && p.g[2] == 1.0 && p.g[3] == 1.0);
    unsigned round = 1;                          // push rounds finished by this CTA
    bool dfresh = true;
    for (long long it = 0; it < nsub; ++it) {
        const long long n = p.reverse ? p.sub_end - 1 - it : p.sub_begin + it;
        const long long tidx = p.reverse ? n + 1 : n;
        if (bound_store && ((tidx - p.sub_begin) % p.bound_step) == 0) {
            S *dst = bound_store + ((size_t)((tidx - p.sub_begin) / p.bound_step) * p.n_states + state) * d2;
            for (int u = u0 + threadIdx.x; u < u1; u += nth)
                store_herm<Num>(dst, d, rc[u - u0].x, rc[u - u0].y, xs[u - u0]);
        }
        const S *A = bands;
        const double *uj = p.u + (size_t)jcur * p.R;
        bool flip = false;
#pragma unroll 1
        for (int s = 0; s < 4; ++s) {
            wait_and_load(round, (round & 1) ? gb0 : gb1);   // round r filled buffer (r - 1) mod 2
            S *nxt = (round & 1) ? gb1 : gb0;
            S *st = nullptr;
            if (stage_store)
                st = stage_store + ((size_t)((n - p.sub_begin) * 4 + p.store_map[s]) * p.n_states + state) * NU;
            const R as_ = ca[s];
#pragma unroll 1
            for (int u = u0 + threadIdx.x; u < u1; u += nth) {
                const int li = u - u0;
                const int2 ij = rc[li];
                const short *na = nbad + (size_t)li * nstride;
                if (st) st[u] = win[na[ns]];
                V dij;
                if (p.fold) {
                    if (s == 0 && dfresh) Dt[li] = Num::store(diag_coef<Num, REALJ>(ij.x, ij.y, d, p.tab, A, vL, vR, uj));
                    dij = Num::load(Dt[li]);
                } else {
                    dij = diag_coef<Num, REALJ>(ij.x, ij.y, d, p.tab, A, vL, vR, uj);
                }
                const V w = lindblad_h_at<Num, REALJ, SH>(win, na, ij.x, ij.y, d, p.tab, A, vL, vR, dij, uj,
                                                      jcache ? jc + li : nullptr, p.cu);
                const V x = Num::load(xs[li]);
                const V acc = Num::axpy(as_, w, s == 0 ? x : Num::load(as[li]));
                V z;
                if (s < 3) {
                    as[li] = Num::store(acc);
                    z = unit_g ? Num::axpy(cb[s + 1], w, x) : Num::lin2(cg[s + 1], x, cb[s + 1], w);
                } else {
                    const V nx = with_source<Num>(p, n, ij.x, ij.y, acc);
                    xs[li] = Num::store(nx);
                    z = Num::scale(cg[0], nx);
                }
                store_herm<Num>(nxt, d, ij.x, ij.y, Num::store(z));
            }
            if (s == 3 && it + 1 < nsub) {
                const long long nn = p.reverse ? n - 1 : n + 1;
                const int jn = (int)(nn / p.n_rk);
                if (jn != jcur) {
                    band_next = jn;
                    jcur = jn;
                    flip = true;
                }
            }
            __syncthreads();
            ++round;
            if (threadIdx.x == 0) {
                __threadfence();
                st_release_gpu(&flags[rank], round);
            }
        }
        dfresh = flip;
    }
    const long long tend = p.reverse ? p.sub_begin : p.sub_end;
    if (bound_store && ((tend - p.sub_begin) % p.bound_step) == 0) {
        S *dst = bound_store + ((size_t)((tend - p.sub_begin) / p.bound_step) * p.n_states + state) * d2;
        for (int u = u0 + threadIdx.x; u < u1; u += nth)
            store_herm<Num>(dst, d, rc[u - u0].x, rc[u - u0].y, xs[u - u0]);
    }
    for (int u = u0 + threadIdx.x; u < u1; u += nth)
        store_herm<Num>(x_out, d, rc[u - u0].x, rc[u - u0].y, xs[u - u0]);
}

// Real-part arithmetic of the trace epilogue in the kernel's own number
// type (double-float on the FP32 pipes, or FP64): the sums never touch the
// FP64 pipe in the double-float build.
__device__ __forceinline__ grape_num::ff r_add(grape_num::ff a, grape_num::ff b) { return grape_num::ff_sum(a, b); }
__device__ __forceinline__ double r_add(double a, double b) { return a + b; }
__device__ __forceinline__ grape_num::ff r_m2(grape_num::ff a) { return {-2.0f * a.h, -2.0f * a.l}; }
__device__ __forceinline__ double r_m2(double a) { return -2.0 * a; }
__device__ __forceinline__ grape_num::ff r_shfl_down(grape_num::ff a, int sh) {
    return {__shfl_down_sync(0xffffffffu, a.h, sh), __shfl_down_sync(0xffffffffu, a.l, sh)};
}
__device__ __forceinline__ double r_shfl_down(double a, int sh) { return __shfl_down_sync(0xffffffffu, a, sh); }
__device__ __forceinline__ double r_double(grape_num::ff a) { return grape_num::ff_to_double(a); }
__device__ __forceinline__ double r_double(double a) { return a; }
__device__ __forceinline__ void r_zero(grape_num::ff &a) { a = {0.0f, 0.0f}; }
__device__ __forceinline__ void r_zero(double &a) { a = 0.0; }

// Epilogue of the trace kernels: per control k, each thread forms
// -2 Im(sum of its band sums of k, in band order) + Re(sum of its sandwich
// sums of k) (ST), the CTA adds the threads by warp shuffles and then the
// warps in index order, all in the number type, and thread k writes
// weight * sum to G (one split) or to its split's partial.  The order is
// fixed by the thread layout alone, so no bit depends on the launch
// grouping or the propagation tile.
template <class Num, bool ST>
__device__ __forceinline__ void trace_store(const TraceArgs &p, typename Num::acc (&Z)[GRAPE_MAXCB],
                                            typename Num::acc (&Zs)[GRAPE_MAXST], int row, int split,
                                            int nwarps = 0) {
    using R = typename Num::real_t;
    __shared__ R redk[GRAPE_MAXR][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (nwarps <= 0) nwarps = blockDim.x >> 5;      // warps whose sums count (in index order)
#pragma unroll
    for (int k = 0; k < GRAPE_MAXR; ++k) {
        if (k >= p.R) break;
        R t;
        r_zero(t);
#pragma unroll
        for (int c = 0; c < GRAPE_MAXCB; ++c)
            if (c < p.ncb && p.cb_k[c] == k) t = r_add(t, Num::im(Num::done(Z[c])));
        R r = r_m2(t);
        if constexpr (ST) {
            R w;
            r_zero(w);
#pragma unroll
            for (int q = 0; q < GRAPE_MAXST; ++q)
                if (q < p.nst && p.st_k[q] == k) w = r_add(w, Num::re(Num::done(Zs[q])));
            r = r_add(r, w);
        }
#pragma unroll
        for (int sh = 16; sh > 0; sh >>= 1) r = r_add(r, r_shfl_down(r, sh));
        if (lane == 0 && warp < nwarps) redk[k][warp] = r;
    }
    __syncthreads();
    if (threadIdx.x < p.R) {
        const int k = threadIdx.x;
        R sum = redk[k][0];
        for (int w = 1; w < nwarps; ++w) sum = r_add(sum, redk[k][w]);
        const double v = p.weight * r_double(sum);
        const int nsplit = max(1, p.nsplit);
        if (nsplit == 1) p.G[(size_t)row * p.R + k] = v;
        else p.part[((size_t)row * nsplit + split) * p.R + k] = v;
    }
}

template <class Num>
__global__ void __launch_bounds__(256) trace_kernel(const TraceArgs p) {
    using S = typename Num::store_t;
    extern __shared__ __align__(16) unsigned char tsmem[];
    S *hv = reinterpret_cast<S *>(tsmem);            // [ncb][d] control band values
    const int nsplit = max(1, p.nsplit);
    const int row = blockIdx.x / nsplit, split = blockIdx.x % nsplit;
    const long long q0 = (long long)split * p.npairs / nsplit;
    const long long q1 = (long long)(split + 1) * p.npairs / nsplit;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int d = p.d;
    const size_t d2 = (size_t)d * d;
    S *svL = hv + p.ncb * d;                         // [nst][d] sandwich tables
    S *svR = svL + p.nst * d;
    for (int i = threadIdx.x; i < p.ncb * d; i += blockDim.x)
        hv[i] = static_cast<const S *>(p.cb_s)[i];
    for (int i = threadIdx.x; i < p.nst * d; i += blockDim.x) {
        svL[i] = static_cast<const S *>(p.st_vLs)[i];
        svR[i] = static_cast<const S *>(p.st_vRs)[i];
    }
    __syncthreads();
    typename Num::acc Z[GRAPE_MAXCB];                // lane-private, in the number type
#pragma unroll
    for (int c = 0; c < GRAPE_MAXCB; ++c) Z[c] = Num::acc_zero();
    typename Num::acc Zs[GRAPE_MAXST];               // sandwich terms (rate controls)
#pragma unroll
    for (int t = 0; t < GRAPE_MAXST; ++t) Zs[t] = Num::acc_zero();
    const S *Kb = static_cast<const S *>(p.K);
    const S *Yb = static_cast<const S *>(p.Y);

#pragma unroll 1
    for (long long q = q0; q < q1; ++q) {
        const size_t moff = ((size_t)row * p.npairs + q) * d2;
        const S *K = Kb + moff;
        const S *Y = Yb + moff;
#pragma unroll 1
        for (int m = warp; m < d; m += nwarps) {
#pragma unroll 1
            for (int o = 0; o < p.ndo; ++o) {
                const int r = m + p.do_off[o];
                if (r < 0 || r >= d) continue;
                typename Num::acc P = Num::acc_zero();
#pragma unroll 1
                for (int l = lane; l < d; l += 32)
                    Num::mac_conjb(P, Num::load(K[(size_t)r * d + l]), Num::load(Y[(size_t)m * d + l]));
                const typename Num::val pv = Num::done(P);
#pragma unroll
                for (int c = 0; c < GRAPE_MAXCB; ++c)
                    if (c < p.ncb && p.cb_do[c] == o) Num::mac(Z[c], Num::load(hv[c * d + m]), pv);
            }
            // rate controls: sum over l of Y[m+oL][l+oR] conj(K[m][l] vR[l]), times vL[m]
#pragma unroll 1
            for (int t = 0; t < p.nst; ++t) {
                const int r = m + p.st_oL[t];
                if (r < 0 || r >= d) continue;
                const int oR = p.st_oR[t];
                typename Num::acc P = Num::acc_zero();
#pragma unroll 1
                for (int l = lane; l < d; l += 32) {
                    const int c = l + oR;
                    if (c < 0 || c >= d) continue;
                    typename Num::acc kv = Num::acc_zero();
                    Num::mac(kv, Num::load(K[(size_t)m * d + l]), Num::load(svR[t * d + l]));
                    Num::mac_conjb(P, Num::load(Y[(size_t)r * d + c]), Num::done(kv));
                }
                Num::mac(Zs[t], Num::load(svL[t * d + m]), Num::done(P));
            }
        }
    }
    trace_store<Num, true>(p, Z, Zs, row, split);
}

// Trace products on packed (upper-triangle) storage, exact gradient.  CTA
// (row, state s, chunk c) takes the upper entries u of its chunk, one per
// thread and pass, and for each distinct control offset o sums over the
// state's pairs (K, Y) of the row, in pair order,
//   S_o(i, j) = sum conj(Y_ij) K_{i+o, j},  T_o(i, j) = sum Y_ij conj(K_{i, j+o})  (i < j)
// (a neighbour below the diagonal is read as the conjugate of its mirror),
// then adds H_o[i] S_o + H_o[j] T_o per control band of that offset:
// Sum over the entries gives Tr(K Y H_k) per pair (see TraceArgs).  The
// rate-control sandwich terms come the same way from
//   conj(K_ij) vL[i] conj(vR[j]) Y_{i+oL, j+oR} + (i < j) K_ij vL[j] conj(vR[i]) Y_{j+oL, i+oR}.
// Lane sums reduce by warp shuffles and a fixed-order tree; the row's
// n_states * nchunk partials are added in order by trace_finish_kernel, so
// no bit depends on the launch grouping or the propagation tile.
template <class Num>
__device__ __forceinline__ typename Num::val conj_if(typename Num::val v, bool c) {
    if (c) v = Num::conj(v);
    return v;
}
__device__ __forceinline__ int packed_index(int r, int c, int d) { return r * d - r * (r - 1) / 2 + (c - r); }

template <class Num>
__global__ void __launch_bounds__(256) trace_packed_kernel(const TraceArgs p) {
    using S = typename Num::store_t;
    using V = typename Num::val;
    const int d = p.d;
    const int NU = d * (d + 1) / 2;
    const int nsplit = p.nsplit;
    const int row = blockIdx.x / nsplit, split = blockIdx.x % nsplit;
    const int state = split / p.nchunk, chunk = split % p.nchunk;
    const long long pps = p.npairs / p.n_states;    // pairs of this state in the row
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const S *Kb = static_cast<const S *>(p.K);
    const S *Yb = static_cast<const S *>(p.Y);
    const S *cbs = static_cast<const S *>(p.cb_s);
    const S *svLs = static_cast<const S *>(p.st_vLs);
    const S *svRs = static_cast<const S *>(p.st_vRs);
    typename Num::acc Z[GRAPE_MAXCB];
#pragma unroll
    for (int c = 0; c < GRAPE_MAXCB; ++c) Z[c] = Num::acc_zero();
    typename Num::acc Zs[GRAPE_MAXST];
#pragma unroll
    for (int t = 0; t < GRAPE_MAXST; ++t) Zs[t] = Num::acc_zero();
    const size_t row_base = (size_t)row * p.npairs;

#pragma unroll 1
    for (int e = 0; e < p.epc; ++e) {
        const int u = (chunk * p.epc + e) * 256 + threadIdx.x;
        if (u >= NU) break;
        const unsigned ij = __ldg(&p.tij[u]);         // row and column of packed entry u
        const int i = (int)(ij & 0xffffu), j = (int)(ij >> 16);
#pragma unroll 1
        for (int oi = 0; oi < p.ndo; ++oi) {
            const int o = p.do_off[oi];
            const int r1 = i + o, c2 = j + o;
            const bool v1 = r1 >= 0 && r1 < d;
            const bool v2 = i < j && c2 >= 0 && c2 < d;
            const bool cj1 = v1 && r1 > j, cj2 = v2 && c2 < i;
            const int x1 = !v1 ? 0 : (cj1 ? packed_index(j, r1, d) : packed_index(r1, j, d));
            const int x2 = !v2 ? 0 : (cj2 ? packed_index(c2, i, d) : packed_index(i, c2, d));
            typename Num::acc Sa = Num::acc_zero(), Ta = Num::acc_zero();
#pragma unroll 1
            for (long long qs = 0; qs < pps; ++qs) {
                const size_t moff = (row_base + (size_t)qs * p.n_states + state) * NU;
                const V y = Num::load(Yb[moff + u]);
                if (v1) Num::mac_conjb(Sa, conj_if<Num>(Num::load(Kb[moff + x1]), cj1), y);
                if (v2) Num::mac_conjb(Ta, y, conj_if<Num>(Num::load(Kb[moff + x2]), cj2));
            }
            const V Sv = Num::done(Sa), Tv = Num::done(Ta);
#pragma unroll
            for (int c = 0; c < GRAPE_MAXCB; ++c) {
                if (c < p.ncb && p.cb_do[c] == oi) {
                    Num::mac(Z[c], Num::load(cbs[c * d + i]), Sv);
                    if (i < j) Num::mac(Z[c], Num::load(cbs[c * d + j]), Tv);
                }
            }
        }
        // rate controls: the sandwich part of Re Tr(kb gamma D[c] y)
#pragma unroll 1
        for (int t = 0; t < p.nst; ++t) {
            const int oL = p.st_oL[t], oR = p.st_oR[t];
            const int ra = i + oL, ca_ = j + oR;            // Y_{i+oL, j+oR}
            const int rb = j + oL, cb_ = i + oR;            // Y_{j+oL, i+oR} (i < j)
            const bool va = ra >= 0 && ra < d && ca_ >= 0 && ca_ < d;
            const bool vb = i < j && rb >= 0 && rb < d && cb_ >= 0 && cb_ < d;
            const bool cja = va && ra > ca_, cjb = vb && rb > cb_;
            const int xa = !va ? 0 : (cja ? packed_index(ca_, ra, d) : packed_index(ra, ca_, d));
            const int xb = !vb ? 0 : (cjb ? packed_index(cb_, rb, d) : packed_index(rb, cb_, d));
            typename Num::acc Pa = Num::acc_zero(), Pb = Num::acc_zero();
#pragma unroll 1
            for (long long qs = 0; qs < pps; ++qs) {
                const size_t moff = (row_base + (size_t)qs * p.n_states + state) * NU;
                const V k = Num::load(Kb[moff + u]);
                if (va) Num::mac_conjb(Pa, conj_if<Num>(Num::load(Yb[moff + xa]), cja), k);   // Y conj(K)
                if (vb) Num::mac(Pb, k, conj_if<Num>(Num::load(Yb[moff + xb]), cjb));        // K Y
            }
            typename Num::acc cL = Num::acc_zero(), cR = Num::acc_zero();
            Num::mac_conjb(cL, Num::load(svLs[t * d + i]),
                           Num::load(svRs[t * d + j]));               // vL[i] conj(vR[j])
            Num::mac_conjb(cR, Num::load(svLs[t * d + j]),
                           Num::load(svRs[t * d + i]));               // vL[j] conj(vR[i])
            Num::mac(Zs[t], Num::done(cL), Num::done(Pa));
            if (vb) Num::mac(Zs[t], Num::done(cR), Num::done(Pb));
        }
    }
    trace_store<Num, true>(p, Z, Zs, row, split);
}

// The same sums for problems without rate-controlled dissipators and with
// at most NDO distinct control offsets: the pairs are the outer loop (each
// Y entry is loaded once per pair) and every offset's sums stay in
// registers.  Each sum adds the same terms in the same order as
// trace_packed_kernel, so both give the same bits.
template <class Num, int NDO>
__global__ void __launch_bounds__(256) trace_packed_fast_kernel(const TraceArgs p) {
    using S = typename Num::store_t;
    using V = typename Num::val;
    const int d = p.d;
    const int NU = d * (d + 1) / 2;
    const int nsplit = p.nsplit;
    const int row = blockIdx.x / nsplit, split = blockIdx.x % nsplit;
    const int state = split / p.nchunk, chunk = split % p.nchunk;
    const long long pps = p.npairs / p.n_states;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const S *Kb = static_cast<const S *>(p.K);
    const S *Yb = static_cast<const S *>(p.Y);
    const S *cbs = static_cast<const S *>(p.cb_s);
    typename Num::acc Z[GRAPE_MAXCB];
#pragma unroll
    for (int c = 0; c < GRAPE_MAXCB; ++c) Z[c] = Num::acc_zero();
    const size_t row_base = (size_t)row * p.npairs;
    const size_t pstride = (size_t)p.n_states * NU;      // between a state's consecutive pairs

#pragma unroll 1
    for (int e = 0; e < p.epc; ++e) {
        const int u = (chunk * p.epc + e) * 256 + threadIdx.x;
        if (u >= NU) break;
        const unsigned ij = __ldg(&p.tij[u]);         // row and column of packed entry u
        const int i = (int)(ij & 0xffffu), j = (int)(ij >> 16);
        int x1[NDO], x2[NDO];
        bool v1[NDO], v2[NDO], cj1[NDO], cj2[NDO];
        typename Num::acc Sa[NDO], Ta[NDO];
#pragma unroll
        for (int oi = 0; oi < NDO; ++oi) {
            const int o = oi < p.ndo ? p.do_off[oi] : 0;
            const int r1 = i + o, c2 = j + o;
            v1[oi] = oi < p.ndo && r1 >= 0 && r1 < d;
            v2[oi] = oi < p.ndo && i < j && c2 >= 0 && c2 < d;
            cj1[oi] = v1[oi] && r1 > j;
            cj2[oi] = v2[oi] && c2 < i;
            x1[oi] = !v1[oi] ? u : (cj1[oi] ? packed_index(j, r1, d) : packed_index(r1, j, d));
            x2[oi] = !v2[oi] ? u : (cj2[oi] ? packed_index(c2, i, d) : packed_index(i, c2, d));
            Sa[oi] = Num::acc_zero();
            Ta[oi] = Num::acc_zero();
        }
        const S *Yp = Yb + (row_base + state) * NU;
        const S *Kp = Kb + (row_base + state) * NU;
#pragma unroll 4
        for (long long qs = 0; qs < pps; ++qs) {
            const size_t moff = (size_t)qs * pstride;
            const V y = Num::load(Yp[moff + u]);
#pragma unroll
            for (int oi = 0; oi < NDO; ++oi) {
                if (v1[oi]) Num::mac_conjb(Sa[oi], conj_if<Num>(Num::load(Kp[moff + x1[oi]]), cj1[oi]), y);
                if (v2[oi]) Num::mac_conjb(Ta[oi], y, conj_if<Num>(Num::load(Kp[moff + x2[oi]]), cj2[oi]));
            }
        }
#pragma unroll
        for (int oi = 0; oi < NDO; ++oi) {
            if (oi >= p.ndo) break;
            const V Sv = Num::done(Sa[oi]), Tv = Num::done(Ta[oi]);
#pragma unroll
            for (int c = 0; c < GRAPE_MAXCB; ++c) {
                if (c < p.ncb && p.cb_do[c] == oi) {
                    Num::mac(Z[c], Num::load(cbs[c * d + i]), Sv);
                    if (i < j) Num::mac(Z[c], Num::load(cbs[c * d + j]), Tv);
                }
            }
        }
    }
    typename Num::acc Z_unused[GRAPE_MAXST];       // no sandwich terms
    trace_store<Num, false>(p, Z, Z_unused, row, split);
}

// The same sums as trace_packed_fast_kernel with the operands staged in
// shared memory by a warp-specialised pipeline.  The CTA of (row, state,
// chunk) walks its 256-entry blocks b = chunk * epc + e and, per block, the
// state's pairs q in order.  Warp 8 is the producer: for each (block, pair)
// step it copies the block's Y entries and the runs of K that hold the
// block's neighbours (host table trun: packed start, length, offset in the
// buffer; gaps of a few entries come along) into one of nbuf buffers with
// bulk asynchronous copies counted on the buffer's "full" mbarrier, after the
// buffer's "empty" mbarrier shows that the eight consumer warps are done with
// its previous use.  Warps 0..7 are the consumers, thread t owning entry
// b * 256 + t: they read its neighbour positions in the buffer from the host
// table tnb (15-bit index, bit 15: read the conjugate of the mirror, 0xffff:
// outside the matrix) and release the buffer warp by warp, so no CTA-wide
// barrier stands between pairs.  Every term and the order of every sum is
// that of the fast kernel: the same bits.  Waits are bounded: one that gives
// up sets the error word to 3 and a shared stop flag, the CTA stops, waits
// (bounded) for the copies it issued and writes no result (the host reports
// GRAPE_ETIMEOUT).
#define GRAPE_TRACE_CONSUMERS 8
#define GRAPE_TRACE_THREADS (32 * (GRAPE_TRACE_CONSUMERS + 1))

// bounded wait that also gives up once *stop is set (by another thread); a
// limit of zero gives up at once, whether or not the phase has completed
__device__ __forceinline__ bool mbar_wait_or_stop(uint32_t mbar, uint32_t parity, long long cycles,
                                                  volatile int *stop) {
    if (cycles <= 0) return false;
    const long long t0 = clock64();
    for (;;) {
        uint32_t done;
        asm volatile("{\n\t.reg .pred p;\n\t"
                     "mbarrier.try_wait.parity.acquire.cta.shared::cta.b64 p, [%1], %2;\n\t"
                     "selp.u32 %0, 1, 0, p;\n\t}"
                     : "=r"(done)
                     : "r"(mbar), "r"(parity)
                     : "memory");
        if (done) return true;
        if (*stop || clock64() - t0 > cycles) return false;
    }
}

template <class Num, int NDO>
__global__ void __launch_bounds__(GRAPE_TRACE_THREADS, 2) trace_tile_kernel(const TraceArgs p) {
    using S = typename Num::store_t;
    using V = typename Num::val;
    using A = typename Num::acc;
    extern __shared__ __align__(128) unsigned char tsm[];
    __shared__ int s_stop;
    const int d = p.d;
    const int NU = d * (d + 1) / 2;
    const int nsplit = p.nsplit;
    const int row = blockIdx.x / nsplit, split = blockIdx.x % nsplit;
    const int state = split / p.nchunk, chunk = split % p.nchunk;
    const int pps = (int)(p.npairs / p.n_states);
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nbuf = p.nbuf;
    const int stride = 256 + p.kcap;                       // entries per buffer: Y block, then K runs
    const uint32_t full0 = (uint32_t)__cvta_generic_to_shared(tsm);     // [nbuf] "full" mbarriers
    const uint32_t empty0 = full0 + 32u;                                // [nbuf] "empty" mbarriers
    A *Zsm = reinterpret_cast<A *>(tsm + 64);                           // [GRAPE_MAXCB][256]
    S *bufs = reinterpret_cast<S *>(tsm + 64 + GRAPE_MAXCB * 256 * sizeof(A));
    const uint32_t ba0 = full0 + 64u + (uint32_t)(GRAPE_MAXCB * 256 * sizeof(A));
    const int nblk_all = (NU + 255) / 256;
    const int b0 = chunk * p.epc;
    const int nblk = max(0, min(p.epc, nblk_all - b0));
    const int total = nblk * pps;
    const size_t row_base = (size_t)row * p.npairs;
    const size_t pstride = (size_t)p.n_states * NU;
    const S *Yp = static_cast<const S *>(p.Y) + (row_base + state) * NU;
    const S *Kp = static_cast<const S *>(p.K) + (row_base + state) * NU;
    const S *cbs = static_cast<const S *>(p.cb_s);
    const long long limit = p.spin;                  // the pipeline's waits
    const long long drain = 1LL << 31;               // waits for copies already issued

    if (tid == 0) {
        for (int b = 0; b < nbuf; ++b) {
            mbar_init(full0 + 8u * b, 1u);
            mbar_init(empty0 + 8u * b, GRAPE_TRACE_CONSUMERS);
        }
        mbar_init_fence();
        s_stop = 0;
    }
    if (tid < 256)
        for (int c = 0; c < GRAPE_MAXCB; ++c) Zsm[c * 256 + tid] = Num::acc_zero();
    __syncthreads();

    int issued = 0;                                  // producer: steps whose copies it issued
    if (warp == GRAPE_TRACE_CONSUMERS) {
        // ---- producer: one step per (block, pair), nbuf - 1 ahead of the slowest consumer
        int buf = 0, use = 0;
        bool stop = false;
        for (int st = 0; st < total && !stop; ++st) {
            const bool ok = use == 0 || mbar_wait_or_stop(empty0 + 8u * buf, (uint32_t)((use - 1) & 1), limit, &s_stop);
            if (!__all_sync(0xffffffffu, ok)) {     // the warp decides as one
                stop = true;
                if (lane == 0) {
                    s_stop = 1;
                    atomicExch(p.err, 3u);
                }
                break;
            }
            const int e = st / pps, q = st - e * pps;
            const int b = b0 + e;
            const int4 bl = __ldg(&p.tblk[b]);             // first run, runs, K entries
            const int ny = min(256, NU - b * 256);
            const uint32_t mb = full0 + 8u * buf;
            const uint32_t dst = ba0 + (uint32_t)(buf * stride) * (uint32_t)sizeof(S);
            const size_t moff = (size_t)q * pstride;
            if (lane == 0) {
                mbar_expect(mb, (uint32_t)(ny + bl.z) * (uint32_t)sizeof(S));
                bulk_g2s(dst, Yp + moff + (size_t)b * 256, (uint32_t)ny * (uint32_t)sizeof(S), mb);
            }
            __syncwarp();
            for (int r = lane; r < bl.y; r += 32) {
                const int4 run = __ldg(&p.trun[bl.x + r]);   // packed start, length, buffer offset
                bulk_g2s(dst + (uint32_t)(256 + run.z) * (uint32_t)sizeof(S), Kp + moff + run.x,
                         (uint32_t)run.y * (uint32_t)sizeof(S), mb);
            }
            ++issued;
            if (++buf == nbuf) {
                buf = 0;
                ++use;
            }
        }
    } else {
        // ---- consumers
        int buf = 0, use = 0;
        bool stop = false;
        const S *Ys = bufs;
#pragma unroll 1
        for (int e = 0; e < nblk && !stop; ++e) {
            const int u = (b0 + e) * 256 + tid;
            const bool valid = u < NU;
            uint4 nb = make_uint4(0xffffffffu, 0xffffffffu, 0xffffffffu, 0xffffffffu);
            unsigned ij = 0u;
            if (valid) {
                nb = __ldg(&p.tnb[u]);
                ij = __ldg(&p.tij[u]);
            }
            const unsigned w16[8] = {nb.x & 0xffffu, nb.x >> 16, nb.y & 0xffffu, nb.y >> 16,
                                     nb.z & 0xffffu, nb.z >> 16, nb.w & 0xffffu, nb.w >> 16};
            int x1[NDO], x2[NDO];
            bool v1[NDO], v2[NDO], cj1[NDO], cj2[NDO];
            A Sa[NDO], Ta[NDO];
#pragma unroll
            for (int oi = 0; oi < NDO; ++oi) {
                const unsigned a = w16[2 * oi], c = w16[2 * oi + 1];
                v1[oi] = valid && a != 0xffffu;
                v2[oi] = valid && c != 0xffffu;
                cj1[oi] = (a & 0x8000u) != 0u;
                cj2[oi] = (c & 0x8000u) != 0u;
                x1[oi] = 256 + (v1[oi] ? (int)(a & 0x7fffu) : 0);
                x2[oi] = 256 + (v2[oi] ? (int)(c & 0x7fffu) : 0);
                Sa[oi] = Num::acc_zero();
                Ta[oi] = Num::acc_zero();
            }
#pragma unroll 1
            for (int q = 0; q < pps; ++q) {
                const bool ok = mbar_wait_or_stop(full0 + 8u * buf, (uint32_t)(use & 1), limit, &s_stop);
                if (!__all_sync(0xffffffffu, ok)) {  // the warp decides as one
                    stop = true;
                    if (lane == 0) {
                        s_stop = 1;
                        atomicExch(p.err, 3u);
                    }
                    break;
                }
                if (valid) {
                    const V y = Num::load(Ys[tid]);
#pragma unroll
                    for (int oi = 0; oi < NDO; ++oi) {
                        if (v1[oi]) Num::mac_conjb(Sa[oi], conj_if<Num>(Num::load(Ys[x1[oi]]), cj1[oi]), y);
                        if (v2[oi]) Num::mac_conjb(Ta[oi], y, conj_if<Num>(Num::load(Ys[x2[oi]]), cj2[oi]));
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(empty0 + 8u * buf);
                if (++buf == nbuf) {
                    buf = 0;
                    ++use;
                    Ys = bufs;
                } else {
                    Ys += stride;
                }
            }
            if (valid && !stop) {
                const int i = (int)(ij & 0xffffu), j = (int)(ij >> 16);
#pragma unroll
                for (int oi = 0; oi < NDO; ++oi) {
                    if (oi >= p.ndo) break;
                    const V Sv = Num::done(Sa[oi]), Tv = Num::done(Ta[oi]);
#pragma unroll
                    for (int c = 0; c < GRAPE_MAXCB; ++c) {
                        if (c < p.ncb && p.cb_do[c] == oi) {
                            A z = Zsm[c * 256 + tid];
                            Num::mac(z, Num::load(cbs[c * d + i]), Sv);
                            if (i < j) Num::mac(z, Num::load(cbs[c * d + j]), Tv);
                            Zsm[c * 256 + tid] = z;
                        }
                    }
                }
            }
        }
    }
    __syncthreads();
    if (s_stop) {
        // a wait gave up somewhere: no CTA leaves while a copy it issued may
        // still write its shared memory (the last nbuf steps' full phases)
        if (warp == GRAPE_TRACE_CONSUMERS && lane == 0)
            for (int st = max(0, issued - nbuf); st < issued; ++st)
                mbar_wait(full0 + 8u * (st % nbuf), (uint32_t)((st / nbuf) & 1), drain);
        __syncthreads();
        return;
    }
    A Z[GRAPE_MAXCB];
#pragma unroll
    for (int c = 0; c < GRAPE_MAXCB; ++c) Z[c] = tid < 256 ? Zsm[c * 256 + tid] : Num::acc_zero();
    A Z_unused[GRAPE_MAXST];                        // no sandwich terms
    trace_store<Num, false>(p, Z, Z_unused, row, split, GRAPE_TRACE_CONSUMERS);
}

// G[row][k] = sum over the row's splits, in split order (deterministic)
static __global__ void __launch_bounds__(256) trace_finish_kernel(const TraceArgs p) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= p.n_rows * p.R) return;
    const int row = idx / p.R, k = idx - row * p.R;
    double s = 0.0;
    for (int sp = 0; sp < p.nsplit; ++sp) s += p.part[((size_t)row * p.nsplit + sp) * p.R + k];
    p.G[(size_t)row * p.R + k] = s;
}

// x[s][i][i] += src[i] (real): the adjoint's start value at the final time
// carries the running cost's last term (App. B)
template <class Num>
__global__ void __launch_bounds__(256) add_diag_kernel(void *x_v, const double *src, int d, int n_states) {
    using S = typename Num::store_t;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= d * n_states) return;
    const int st = idx / d, i = idx - st * d;
    S *x = static_cast<S *>(x_v) + (size_t)st * d * d + (size_t)i * d + i;
    *x = Num::store(Num::add_real(Num::load(*x), Num::real_const(src[i])));
}

// out[row] = sum over states and i of diag[i] Re x_row[s][i][i], states then
// rows in index order (FP64); x_row = x + row * row_stride entries
// (packed: the states are upper triangles of d(d+1)/2 entries)
template <class Num>
__global__ void __launch_bounds__(128) penalty_rows_kernel(const void *x_v, long long row_stride, int rows,
                                                           int n_states, int d, const double *diag,
                                                           double *out, int packed) {
    using S = typename Num::store_t;
    const int row = blockIdx.x * blockDim.x + threadIdx.x;
    if (row >= rows) return;
    const S *x = static_cast<const S *>(x_v) + (size_t)row * row_stride;
    const size_t m = packed ? (size_t)d * (d + 1) / 2 : (size_t)d * d;
    double acc = 0.0;
    for (int st = 0; st < n_states; ++st)
        for (int i = 0; i < d; ++i) {
            const size_t ii = packed ? (size_t)packed_index(i, i, d) : (size_t)i * d + i;
            acc = fma(diag[i], Num::to_double2(Num::load(x[st * m + ii])).x, acc);
        }
    out[row] = acc;
}

// F -= scale * sum_k pen[k], in index order (one thread: deterministic)
static __global__ void penalty_finish_kernel(const double *pen, long long count, double scale, double *F) {
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    double t = 0.0;
    for (long long k = 0; k < count; ++k) t += pen[k];
    F[0] -= scale * t;
}

template <class Num>
__global__ void __launch_bounds__(256) cost_kernel(const void *rho_v, const void *sigma_v,
                                                   int n_states, int d2, double *F) {
    using S = typename Num::store_t;
    const S *rho = static_cast<const S *>(rho_v);
    const S *sigma = static_cast<const S *>(sigma_v);
    double acc = 0.0;
    for (int s = 0; s < n_states; ++s)
        for (int e = threadIdx.x; e < d2; e += blockDim.x) {
            const double2 r = Num::to_double2(Num::load(rho[(size_t)s * d2 + e]));
            const double2 g = Num::to_double2(Num::load(sigma[(size_t)s * d2 + e]));
            acc = fma(g.x, r.x, fma(g.y, r.y, acc));    // Re(conj(sigma_ij) rho_ij)
        }
#pragma unroll
    for (int sh = 16; sh > 0; sh >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, sh);
    __shared__ double red[32];
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
        *F = s;
    }
}

template <class Num>
__global__ void __launch_bounds__(256) to_double_kernel(const void *src_v, double2 *dst, size_t n) {
    using S = typename Num::store_t;
    const S *src = static_cast<const S *>(src_v);
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n;
         i += (size_t)gridDim.x * blockDim.x)
        dst[i] = Num::to_double2(Num::load(src[i]));
}

// ------------------------------------------------------------------ launchers
// `variant`: bit 0 the jump tables are real; bit 1 Hermitian (upper-triangle)
// kernel; bits 2-3 the band/jump shape (0 from the tables, 1 ShapeT, 2 ShapeR;
// only with real jump tables); bit 4 one entry per thread (with a shape).
using PropKernel = void (*)(const PropArgs);

template <class Num>
PropKernel prop_kernel_for(int variant) {
    const bool realj = (variant & 1) != 0, herm = (variant & 2) != 0, one = (variant & 16) != 0;
    const int shape = (variant >> 2) & 3;
    if (!herm) return realj ? prop_kernel<Num, true> : prop_kernel<Num, false>;
    if (realj && shape == 1) return one ? prop_h_kernel<Num, true, ShapeT, true> : prop_h_kernel<Num, true, ShapeT, false>;
    if (realj && shape == 2) return one ? prop_h_kernel<Num, true, ShapeR, true> : prop_h_kernel<Num, true, ShapeR, false>;
    return realj ? prop_h_kernel<Num, true, ShapeAny, false> : prop_h_kernel<Num, false, ShapeAny, false>;
}

template <class Num>
PropKernel grid_kernel_for(int variant) {
    const bool realj = (variant & 1) != 0;
    const int shape = (variant >> 2) & 3;
    if (realj && shape == 1) return prop_g_kernel<Num, true, ShapeT>;
    if (realj && shape == 2) return prop_g_kernel<Num, true, ShapeR>;
    return realj ? prop_g_kernel<Num, true, ShapeAny> : prop_g_kernel<Num, false, ShapeAny>;
}

template <class Num>
cudaError_t launch_prop(const PropArgs &p, int threads, int variant, size_t smem, cudaStream_t stream) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(p.n_states * p.ncl));
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)p.ncl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, prop_kernel_for<Num>(variant), p);
}

// smem_total: the per-block shared-memory budget; the dynamic limit is that
// budget minus the kernel's static shared memory.
template <typename K>
cudaError_t prepare_kernel(K kernel, size_t smem_total, int ncl) {
    cudaFuncAttributes fa;
    cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
    if (e != cudaSuccess) return e;
    if (fa.sharedSizeBytes > smem_total) return cudaErrorInvalidValue;
    e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)(smem_total - fa.sharedSizeBytes));
    if (e != cudaSuccess) return e;
    if (ncl > 8) e = cudaFuncSetAttribute(kernel, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

template <class Num>
cudaError_t prepare(int variant, size_t smem, int ncl) {
    return prepare_kernel(prop_kernel_for<Num>(variant), smem, ncl);
}

template <class Num>
cudaError_t max_clusters(int threads, int variant, size_t smem, int ncl, int n_blocks, int *clusters) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)n_blocks);
    cfg.blockDim = dim3((unsigned)threads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)ncl;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaOccupancyMaxActiveClusters(clusters, prop_kernel_for<Num>(variant), &cfg);
}

template <class Num>
cudaError_t launch_grid(const PropArgs &p, int nblocks, int variant, size_t smem, cudaStream_t stream) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)nblocks);
    cfg.blockDim = dim3(GRAPE_GRID_THREADS);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, grid_kernel_for<Num>(variant), p);
}

// prepares the grid kernel and returns how many CTAs of it fit on the device at once
template <class Num>
cudaError_t prepare_grid(int variant, size_t smem_total, size_t smem, int *max_blocks) {
    const PropKernel k = grid_kernel_for<Num>(variant);
    cudaError_t e = prepare_kernel(k, smem_total, 1);
    if (e != cudaSuccess) return e;
    int per_sm = 0, dev = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, GRAPE_GRID_THREADS, smem);
    if (e != cudaSuccess) return e;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    *max_blocks = per_sm * sms;
    return cudaSuccess;
}

template <class Num>
cudaError_t launch_trace(const TraceArgs &p, cudaStream_t s) {
    if (p.n_rows <= 0) return cudaSuccess;
    if (p.packed) {
        const int grid = p.n_rows * max(1, p.nsplit);
        if (p.tile && p.nst == 0 && p.ndo <= 4) {
            const size_t smem = trace_tile_smem(p.nbuf, p.kcap);
            void (*k)(const TraceArgs) = p.ndo <= 2 ? trace_tile_kernel<Num, 2> : trace_tile_kernel<Num, 4>;
            const cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            k<<<grid, GRAPE_TRACE_THREADS, smem, s>>>(p);
        } else if (p.nst == 0 && p.ndo <= 2) trace_packed_fast_kernel<Num, 2><<<grid, 256, 0, s>>>(p);
        else if (p.nst == 0 && p.ndo <= 4) trace_packed_fast_kernel<Num, 4><<<grid, 256, 0, s>>>(p);
        else trace_packed_kernel<Num><<<grid, 256, 0, s>>>(p);
        return cudaGetLastError();
    }
    const size_t smem = (size_t)(p.ncb + 2 * p.nst) * p.d * sizeof(typename Num::store_t);
    if (smem > 48 * 1024) {
        const cudaError_t e = cudaFuncSetAttribute(trace_kernel<Num>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    trace_kernel<Num><<<p.n_rows * max(1, p.nsplit), 256, smem, s>>>(p);
    return cudaGetLastError();
}

static cudaError_t launch_trace_finish(const TraceArgs &p, cudaStream_t s) {
    if (p.n_rows <= 0 || p.nsplit <= 1) return cudaSuccess;
    const int n = p.n_rows * p.R;
    trace_finish_kernel<<<(n + 255) / 256, 256, 0, s>>>(p);
    return cudaGetLastError();
}

template <class Num>
cudaError_t launch_cost(const void *rho, const void *sigma, int n_states, int d2, double *F,
                        cudaStream_t s) {
    cost_kernel<Num><<<1, 256, 0, s>>>(rho, sigma, n_states, d2, F);
    return cudaGetLastError();
}

template <class Num>
cudaError_t launch_to_double(const void *src, double2 *dst, size_t n, cudaStream_t s) {
    const int blocks = (int)std::min<size_t>((n + 255) / 256, 1024);
    if (blocks <= 0) return cudaSuccess;
    to_double_kernel<Num><<<blocks, 256, 0, s>>>(src, dst, n);
    return cudaGetLastError();
}

template <class Num>
cudaError_t launch_add_diag(void *x, const double *src, int d, int ns, cudaStream_t s) {
    add_diag_kernel<Num><<<(d * ns + 255) / 256, 256, 0, s>>>(x, src, d, ns);
    return cudaGetLastError();
}
template <class Num>
cudaError_t launch_penalty_rows(const void *x, long long stride, int rows, int ns, int d,
                                const double *diag, double *out, int packed, cudaStream_t s) {
    if (rows <= 0) return cudaSuccess;
    penalty_rows_kernel<Num><<<(rows + 127) / 128, 128, 0, s>>>(x, stride, rows, ns, d, diag, out, packed);
    return cudaGetLastError();
}
static cudaError_t launch_penalty_finish(const double *pen, long long count, double scale, double *F,
                                         cudaStream_t s) {
    penalty_finish_kernel<<<1, 32, 0, s>>>(pen, count, scale, F);
    return cudaGetLastError();
}

}  // namespace grape_k

#define GRAPE_DEFINE_LAUNCHERS(SUFFIX, NUM)                                                     \
    cudaError_t grape_launch_prop_##SUFFIX(const PropArgs &p, int threads, int variant,         \
                                           size_t smem, cudaStream_t s) {                       \
        return grape_k::launch_prop<NUM>(p, threads, variant, smem, s);                         \
    }                                                                                           \
    cudaError_t grape_prepare_prop_##SUFFIX(int variant, size_t smem, int ncl) {                \
        return grape_k::prepare<NUM>(variant, smem, ncl);                                       \
    }                                                                                           \
    cudaError_t grape_max_active_clusters_##SUFFIX(int threads, int variant, size_t smem,       \
                                                   int ncl, int n_blocks, int *clusters) {      \
        return grape_k::max_clusters<NUM>(threads, variant, smem, ncl, n_blocks, clusters);     \
    }                                                                                           \
    cudaError_t grape_launch_trace_##SUFFIX(const TraceArgs &p, cudaStream_t s) {               \
        return grape_k::launch_trace<NUM>(p, s);                                                \
    }                                                                                           \
    cudaError_t grape_launch_trace_finish_##SUFFIX(const TraceArgs &p, cudaStream_t s) {        \
        return grape_k::launch_trace_finish(p, s);                                              \
    }                                                                                           \
    cudaError_t grape_launch_cost_##SUFFIX(const void *rho, const void *sigma, int n_states,    \
                                           int d2, double *F, cudaStream_t s) {                 \
        return grape_k::launch_cost<NUM>(rho, sigma, n_states, d2, F, s);                       \
    }                                                                                           \
    cudaError_t grape_launch_to_double_##SUFFIX(const void *src, double2 *dst, size_t n,        \
                                                cudaStream_t s) {                               \
        return grape_k::launch_to_double<NUM>(src, dst, n, s);                                  \
    }                                                                                           \
    cudaError_t grape_launch_grid_##SUFFIX(const PropArgs &p, int nblocks, int variant,         \
                                           size_t smem, cudaStream_t s) {                       \
        return grape_k::launch_grid<NUM>(p, nblocks, variant, smem, s);                         \
    }                                                                                           \
    cudaError_t grape_prepare_grid_##SUFFIX(int variant, size_t smem_total, size_t smem,        \
                                            int *max_blocks) {                                  \
        return grape_k::prepare_grid<NUM>(variant, smem_total, smem, max_blocks);               \
    }                                                                                           \
    cudaError_t grape_launch_add_diag_##SUFFIX(void *x, const double *src, int d, int n_states, \
                                               cudaStream_t s) {                                \
        return grape_k::launch_add_diag<NUM>(x, src, d, n_states, s);                           \
    }                                                                                           \
    cudaError_t grape_launch_penalty_rows_##SUFFIX(const void *x, long long row_stride, int rows, \
                                                   int n_states, int d, const double *diag,     \
                                                   double *out, int packed, cudaStream_t s) {   \
        return grape_k::launch_penalty_rows<NUM>(x, row_stride, rows, n_states, d, diag, out,   \
                                                 packed, s);                                    \
    }                                                                                           \
    cudaError_t grape_launch_penalty_finish_##SUFFIX(const double *pen, long long count,        \
                                                     double scale, double *F, cudaStream_t s) {  \
        return grape_k::launch_penalty_finish(pen, count, scale, F, s);                         \
    }
