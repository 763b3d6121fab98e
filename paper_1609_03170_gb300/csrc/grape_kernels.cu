// grape_kernels.cu - sm_103a kernels of the open-GRAPE hot path.
//
//  prop_kernel   RK4 propagation of one density matrix (forward, Sec. 3
//                Eq. rkmaster) or of its adjoint (backward, Eq. lambda) per
//                thread-block cluster.  The d x d matrix is split into
//                contiguous chunks of its row-major flat index, one per CTA
//                of the cluster.  Each CTA keeps the current stage input of
//                its chunk plus a halo of omax*(d+1) entries on both sides in
//                shared memory; new stage values are pushed into the
//                neighbours' halos with distributed-shared-memory stores and
//                one cluster barrier separates consecutive RK stages.  The
//                slice's Hamiltonian bands A(u_j) are rebuilt in shared
//                memory once per slice.  Stage inputs (forward y_s, adjoint
//                kb_s) and slice-boundary states are streamed to HBM for the
//                gradient.
//  trace_kernel  per-slice gradient reduction of Eq. (dphidu): one CTA per
//                slice, row dot-products of K and conj(Y) on the control
//                bands, lane-private accumulation, warp-shuffle plus a
//                fixed-order shared-memory tree (deterministic).
//  cost_kernel   Phi = sum_s Re Tr(sigma_s rho_s(T)) (Eq. phi), fixed order.
#include "grape_internal.h"

namespace {

__device__ __forceinline__ void cfma(double2 &acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, fma(-a.y, b.y, acc.x));
    acc.y = fma(a.x, b.y, fma(a.y, b.x, acc.y));
}
// acc -= conj(a) * b
__device__ __forceinline__ void cfms_conja(double2 &acc, double2 a, double2 b) {
    acc.x = fma(-a.x, b.x, fma(-a.y, b.y, acc.x));
    acc.y = fma(-a.x, b.y, fma(a.y, b.x, acc.y));
}
// a * conj(b)
__device__ __forceinline__ double2 cmul_conjb(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, a.y * b.y), fma(a.y, b.x, -a.x * b.y));
}
// acc += a * conj(b)
__device__ __forceinline__ void cfma_conjb(double2 &acc, double2 a, double2 b) {
    acc.x = fma(a.x, b.x, fma(a.y, b.y, acc.x));
    acc.y = fma(a.y, b.x, fma(-a.x, b.y, acc.y));
}

__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\t"
                 "barrier.cluster.wait.acquire.aligned;" ::: "memory");
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

// A(u_j) = A0 + sum_k u_k(j) Ak into shared memory.
__device__ __forceinline__ void build_bands(double2 *dst, const PropArgs &p, int slice) {
    const int nbd = p.tab.nb * p.d;
    const double *uj = p.u + (size_t)slice * p.R;
    for (int idx = threadIdx.x; idx < nbd; idx += blockDim.x) {
        double2 v = __ldg(&p.tab.A0[idx]);
        for (int k = 0; k < p.R; ++k) {
            const double uk = __ldg(&uj[k]);
            const double2 h = __ldg(&p.tab.Ak[(size_t)k * nbd + idx]);
            v.x = fma(uk, h.x, v.x);
            v.y = fma(uk, h.y, v.y);
        }
        dst[idx] = v;
    }
}

// Write stage value z of flat element e into the own window and into every
// neighbour window of the cluster that covers e.
__device__ __forceinline__ void push_value(double2 *buf, const PropArgs &p, int rank, int e,
                                           double2 z) {
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

// W = Op(z) at element (i, j) of the window `cur` (local flat index le).
__device__ __forceinline__ double2 lindblad_at(const double2 *cur, int le, int i, int j, int d,
                                               const PropTables &t, const double2 *A,
                                               const double2 *vL, const double2 *vR) {
    double2 w = make_double2(0.0, 0.0);
#pragma unroll
    for (int b = 0; b < GRAPE_MAXB; ++b) {
        if (b < t.nb) {
            const double2 ai = A[b * d + i];
            const double2 aj = A[b * d + j];
            cfma(w, ai, cur[le + t.off_row[b]]);       // (A X)[i][j]
            cfms_conja(w, aj, cur[le + t.off[b]]);     // -(X A^+)[i][j]
        }
    }
    double2 out = make_double2(w.y, -w.x);             // -i * w
#pragma unroll
    for (int q = 0; q < GRAPE_MAXT; ++q) {
        if (q < t.nt) {
            const double2 coef = cmul_conjb(vL[q * d + i], vR[q * d + j]);
            cfma(out, coef, cur[le + t.jflat[q]]);
        }
    }
    return out;
}

template <int EPT>
__global__ void __launch_bounds__(256) prop_kernel(const PropArgs p) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    double2 *buf0 = reinterpret_cast<double2 *>(smem_raw);
    double2 *buf1 = buf0 + p.win;
    const int d = p.d, d2 = d * d;
    const int nbd = p.tab.nb * d;
    double2 *bands = buf1 + p.win;                 // [2][nb][d]
    double2 *vL = bands + 2 * nbd;                 // [nt][d]
    double2 *vR = vL + p.tab.nt * d;               // [nt][d]

    const int rank = blockIdx.x % p.ncl;
    const int state = blockIdx.x / p.ncl;
    const int e0 = rank * p.chunk;
    const int e1 = min(e0 + p.chunk, d2);
    const int wbase = e0 - p.halo;
    const size_t soff = (size_t)state * d2;

    for (int i = threadIdx.x; i < 2 * p.win; i += blockDim.x) buf0[i] = make_double2(0.0, 0.0);
    for (int i = threadIdx.x; i < p.tab.nt * d; i += blockDim.x) {
        vL[i] = __ldg(&p.tab.vL[i]);
        vR[i] = __ldg(&p.tab.vR[i]);
    }
    const long long nsub = p.sub_end - p.sub_begin;
    long long n_first = p.reverse ? p.sub_end - 1 : p.sub_begin;
    if (nsub <= 0) n_first = p.sub_begin;
    int jcur = (int)(n_first / p.n_rk);
    build_bands(bands, p, jcur);
    cluster_sync_all();   // every CTA of the cluster runs and has zeroed its windows

    double2 x[EPT], acc[EPT];
    int el[EPT], ri[EPT], ci[EPT];
#pragma unroll
    for (int k = 0; k < EPT; ++k) {
        const int e = e0 + threadIdx.x + k * blockDim.x;
        el[k] = (e < e1) ? e : -1;
        ri[k] = (e < e1) ? e / d : 0;
        ci[k] = (e < e1) ? e - (e / d) * d : 0;
        x[k] = (e < e1) ? p.x_in[soff + e] : make_double2(0.0, 0.0);
        if (e < e1) push_value(buf0, p, rank, e, make_double2(p.g[0] * x[k].x, p.g[0] * x[k].y));
    }
    cluster_sync_all();

    int tb = 0;
    for (long long it = 0; it < nsub; ++it) {
        const long long n = p.reverse ? p.sub_end - 1 - it : p.sub_begin + it;
        const long long tidx = p.reverse ? n + 1 : n;
        if (p.bound_store && ((tidx - p.sub_begin) % p.bound_step) == 0) {
            double2 *dst = p.bound_store +
                           ((size_t)((tidx - p.sub_begin) / p.bound_step) * p.n_states) * d2 + soff;
#pragma unroll
            for (int k = 0; k < EPT; ++k)
                if (el[k] >= 0) dst[el[k]] = x[k];
        }
#pragma unroll
        for (int k = 0; k < EPT; ++k) acc[k] = x[k];
        const double2 *A = bands + tb * nbd;
        bool flip = false;
#pragma unroll
        for (int s = 0; s < 4; ++s) {
            const double2 *cur = (s & 1) ? buf1 : buf0;
            double2 *nxt = (s & 1) ? buf0 : buf1;
            double2 *st = nullptr;
            if (p.stage_store)
                st = p.stage_store +
                     ((size_t)((n - p.sub_begin) * 4 + p.store_map[s]) * p.n_states) * d2 + soff;
#pragma unroll
            for (int k = 0; k < EPT; ++k) {
                if (el[k] < 0) continue;
                const int le = el[k] - wbase;
                const double2 w = lindblad_at(cur, le, ri[k], ci[k], d, p.tab, A, vL, vR);
                if (st) st[el[k]] = cur[le];
                acc[k].x = fma(p.a[s], w.x, acc[k].x);
                acc[k].y = fma(p.a[s], w.y, acc[k].y);
                double2 z;
                if (s < 3) {
                    z.x = fma(p.g[s + 1], x[k].x, p.b[s + 1] * w.x);
                    z.y = fma(p.g[s + 1], x[k].y, p.b[s + 1] * w.y);
                } else {
                    x[k] = acc[k];
                    z.x = p.g[0] * x[k].x;
                    z.y = p.g[0] * x[k].y;
                }
                push_value(nxt, p, rank, el[k], z);
            }
            if (s == 3 && it + 1 < nsub) {
                const long long nn = p.reverse ? n - 1 : n + 1;
                const int jn = (int)(nn / p.n_rk);
                if (jn != jcur) {
                    build_bands(bands + (tb ^ 1) * nbd, p, jn);
                    jcur = jn;
                    flip = true;
                }
            }
            cluster_sync_all();
        }
        if (flip) tb ^= 1;
    }
    const long long tend = p.reverse ? p.sub_begin : p.sub_end;
    if (p.bound_store && ((tend - p.sub_begin) % p.bound_step) == 0) {
        double2 *dst = p.bound_store +
                       ((size_t)((tend - p.sub_begin) / p.bound_step) * p.n_states) * d2 + soff;
#pragma unroll
        for (int k = 0; k < EPT; ++k)
            if (el[k] >= 0) dst[el[k]] = x[k];
    }
#pragma unroll
    for (int k = 0; k < EPT; ++k)
        if (el[k] >= 0) p.x_out[soff + el[k]] = x[k];
}

__global__ void __launch_bounds__(256) trace_kernel(const TraceArgs p) {
    const int row = blockIdx.x;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const int d = p.d;
    const size_t d2 = (size_t)d * d;
    double2 Z[GRAPE_MAXCB];
#pragma unroll
    for (int c = 0; c < GRAPE_MAXCB; ++c) Z[c] = make_double2(0.0, 0.0);

    for (long long q = 0; q < p.npairs; ++q) {
        const size_t moff = ((size_t)row * p.npairs + q) * d2;
        const double2 *K = p.K + moff;
        const double2 *Y = p.Y + moff;
        for (int m = warp; m < d; m += nwarps) {
            double2 P[GRAPE_MAXDO];
#pragma unroll
            for (int o = 0; o < GRAPE_MAXDO; ++o) P[o] = make_double2(0.0, 0.0);
            for (int l = lane; l < d; l += 32) {
                const double2 y = __ldg(&Y[(size_t)m * d + l]);
#pragma unroll
                for (int o = 0; o < GRAPE_MAXDO; ++o) {
                    if (o < p.ndo) {
                        const int r = m + p.do_off[o];
                        if (r >= 0 && r < d) cfma_conjb(P[o], __ldg(&K[(size_t)r * d + l]), y);
                    }
                }
            }
#pragma unroll
            for (int c = 0; c < GRAPE_MAXCB; ++c) {
                if (c < p.ncb) {
                    const double2 hv = __ldg(&p.cb_val[(size_t)c * d + m]);
#pragma unroll
                    for (int o = 0; o < GRAPE_MAXDO; ++o)
                        if (o == p.cb_do[c]) cfma(Z[c], hv, P[o]);
                }
            }
        }
    }
    // deterministic reduction: warp shuffles, then warps in index order
    __shared__ double red[GRAPE_MAXCB][32];
#pragma unroll
    for (int c = 0; c < GRAPE_MAXCB; ++c) {
        double v = Z[c].y;
#pragma unroll
        for (int sh = 16; sh > 0; sh >>= 1) v += __shfl_down_sync(0xffffffffu, v, sh);
        if (lane == 0) red[c][warp] = v;
    }
    __syncthreads();
    if (threadIdx.x < GRAPE_MAXR) {
        const int k = threadIdx.x;
        if (k < p.R) {
            double s = 0.0;
            for (int c = 0; c < p.ncb; ++c) {
                if (p.cb_k[c] != k) continue;
                double t = 0.0;
                for (int w = 0; w < nwarps; ++w) t += red[c][w];
                s += t;
            }
            p.G[(size_t)row * p.R + k] = p.weight * (-2.0 * s);
        }
    }
}

__global__ void __launch_bounds__(256) cost_kernel(const double2 *rho, const double2 *sigma,
                                                   int n_states, int d2, double *F) {
    double acc = 0.0;
    for (int s = 0; s < n_states; ++s)
        for (int e = threadIdx.x; e < d2; e += blockDim.x) {
            const double2 r = rho[(size_t)s * d2 + e], g = sigma[(size_t)s * d2 + e];
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

template <int EPT>
cudaError_t launch_prop_t(const PropArgs &p, int threads, size_t smem, cudaStream_t stream) {
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
    return cudaLaunchKernelEx(&cfg, prop_kernel<EPT>, p);
}

template <int EPT>
cudaError_t prepare_t(size_t smem, int ncl) {
    cudaError_t e = cudaFuncSetAttribute(prop_kernel<EPT>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    if (ncl > 8)
        e = cudaFuncSetAttribute(prop_kernel<EPT>,
                                 cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    return e;
}

template <int EPT>
cudaError_t clusters_t(int threads, size_t smem, int ncl, int n_blocks, int *clusters) {
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
    return cudaOccupancyMaxActiveClusters(clusters, prop_kernel<EPT>, &cfg);
}

}  // namespace

cudaError_t grape_launch_prop(const PropArgs &p, int threads, int ept, size_t smem,
                              cudaStream_t stream) {
    switch (ept) {
    case 1: return launch_prop_t<1>(p, threads, smem, stream);
    case 2: return launch_prop_t<2>(p, threads, smem, stream);
    case 4: return launch_prop_t<4>(p, threads, smem, stream);
    case 8: return launch_prop_t<8>(p, threads, smem, stream);
    case 16: return launch_prop_t<16>(p, threads, smem, stream);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t grape_prepare_prop(int ept, size_t smem, int ncl) {
    switch (ept) {
    case 1: return prepare_t<1>(smem, ncl);
    case 2: return prepare_t<2>(smem, ncl);
    case 4: return prepare_t<4>(smem, ncl);
    case 8: return prepare_t<8>(smem, ncl);
    case 16: return prepare_t<16>(smem, ncl);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t grape_max_active_clusters(int threads, int ept, size_t smem, int ncl, int n_blocks,
                                      int *clusters) {
    switch (ept) {
    case 1: return clusters_t<1>(threads, smem, ncl, n_blocks, clusters);
    case 2: return clusters_t<2>(threads, smem, ncl, n_blocks, clusters);
    case 4: return clusters_t<4>(threads, smem, ncl, n_blocks, clusters);
    case 8: return clusters_t<8>(threads, smem, ncl, n_blocks, clusters);
    case 16: return clusters_t<16>(threads, smem, ncl, n_blocks, clusters);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t grape_launch_trace(const TraceArgs &p, cudaStream_t stream) {
    if (p.n_rows <= 0) return cudaSuccess;
    trace_kernel<<<p.n_rows, 256, 0, stream>>>(p);
    return cudaGetLastError();
}

cudaError_t grape_launch_cost(const double2 *rho, const double2 *sigma, int n_states, int d2,
                              double *F, cudaStream_t stream) {
    cost_kernel<<<1, 256, 0, stream>>>(rho, sigma, n_states, d2, F);
    return cudaGetLastError();
}
