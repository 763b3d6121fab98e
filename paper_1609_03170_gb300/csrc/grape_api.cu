// grape_api.cu - C ABI of libgrape.so (declared in include/grape.h).
//
// Host-side work: validation of the problem descriptor, band (DIA) algebra
// that turns H_0, H_k and the jump operators into the two kernel tables
// (forward Lindbladian, Eq. master/disspation, and its dual), the launch
// geometry, the segment plan of the gradient (stage storage or checkpoints
// plus recomputation) and the launch sequence of grape_forward and
// grape_gradient.  All arithmetic of the propagation and of the gradient
// runs in the kernels of grape_kernels.cuh (instantiated per number type by
// grape_kernels_df.cu and grape_kernels_f64.cu).
#include "grape.h"
#include "grape_internal.h"
#include "grape_num.cuh"

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <condition_variable>
#include <deque>
#include <mutex>
#include <thread>
#include <complex>
#include <cstdlib>
#include <cstring>
#include <map>
#include <climits>
#include <cstdint>
#include <string>
#include <vector>

// Looks up the device address of the no-allocation entry point's static
// scratch array once per device (defined with the array, further below).
static void static_scratch_setup(int dev);

namespace {

using cplx = std::complex<double>;
using Bands = std::map<int, std::vector<cplx>>;   // offset o -> Op[i][i+o], i in [0, d)

thread_local std::string g_last_error;

grape_status fail(grape_status s, const std::string &msg) {
    g_last_error = msg;
    return s;
}

#define GRAPE_CUDA_TRY(expr)                                                              \
    do {                                                                                  \
        cudaError_t e_ = (expr);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(GRAPE_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
    } while (0)

bool valid_entry(int i, int o, int d) { return i + o >= 0 && i + o < d; }

grape_status read_bands(const grape_band_op &op, int d, const char *name, Bands *out) {
    Bands B;
    if (op.n_diag < 0 || (op.n_diag > 0 && (!op.offsets || !op.values)))
        return fail(GRAPE_EINVAL, std::string(name) + ": bad band list");
    for (int b = 0; b < op.n_diag; ++b) {
        const int o = op.offsets[b];
        if (o <= -d || o >= d) return fail(GRAPE_EINVAL, std::string(name) + ": band offset out of range");
        auto &v = B[o];
        v.resize(d);
        for (int i = 0; i < d; ++i) {
            if (!valid_entry(i, o, d)) continue;   // entries outside the matrix are ignored
            const double re = op.values[2 * ((size_t)b * d + i)];
            const double im = op.values[2 * ((size_t)b * d + i) + 1];
            if (!std::isfinite(re) || !std::isfinite(im))
                return fail(GRAPE_EINVAL, std::string(name) + ": non-finite value");
            v[i] += cplx(re, im);
        }
    }
    *out = B;
    return GRAPE_OK;
}

void add_into(Bands &dst, const Bands &src, cplx s, int d) {
    for (const auto &kv : src) {
        auto &v = dst[kv.first];
        v.resize(d);
        for (int i = 0; i < d; ++i) v[i] += s * kv.second[i];
    }
}

Bands adjoint(const Bands &A, int d) {
    Bands R;
    for (const auto &kv : A) {
        const int o = kv.first;
        auto &w = R[-o];
        w.resize(d);
        for (int i = 0; i < d; ++i)
            if (i - o >= 0 && i - o < d) w[i] = std::conj(kv.second[i - o]);   // A^+[i][i-o] = conj(A[i-o][i])
    }
    return R;
}

Bands product(const Bands &A, const Bands &B, int d) {
    Bands R;
    for (const auto &a : A)
        for (const auto &b : B) {
            const int o = a.first + b.first;
            if (o <= -d || o >= d) continue;
            auto &w = R[o];
            w.resize(d);
            for (int i = 0; i < d; ++i) {
                const int m = i + a.first;
                if (m < 0 || m >= d || !valid_entry(m, b.first, d)) continue;
                w[i] += a.second[i] * b.second[m];
            }
        }
    return R;
}

Bands scaled(const Bands &A, cplx s, int d) {
    Bands R;
    add_into(R, A, s, d);
    return R;
}

void prune(Bands &A) {
    for (auto it = A.begin(); it != A.end();) {
        bool zero = true;
        for (const cplx &c : it->second)
            if (c != cplx(0.0, 0.0)) { zero = false; break; }
        it = zero ? A.erase(it) : std::next(it);
    }
}

double max_abs(const Bands &A) {
    double m = 0.0;
    for (const auto &kv : A)
        for (const cplx &c : kv.second) m = std::max(m, std::abs(c));
    return m;
}

bool hermitian(const Bands &A, int d) {
    Bands D = A;
    add_into(D, adjoint(A, d), -1.0, d);
    return max_abs(D) <= 1e-12 * std::max(1.0, max_abs(A));
}

struct HostDir {
    std::vector<int> off;        // nb
    int nbr = 0;                 // leading bands that are real for every control value
    std::vector<cplx> A0, Ak;    // [nb][d], [R][nb][d]
    std::vector<int> oL, oR;     // nt
    std::vector<cplx> vL, vR;    // [nt][d]
    std::vector<int> jctl;       // nt: control scaling the term, -1 fixed
};

HostDir make_dir(const Bands &A0, const std::vector<Bands> &Ak,
                 const std::vector<Bands> &jumps, const std::vector<int> &jump_ctl, int d) {
    HostDir h;
    std::map<int, int> idx;
    for (const auto &kv : A0) idx[kv.first] = 0;
    for (const auto &B : Ak)
        for (const auto &kv : B) idx[kv.first] = 0;
    // bands whose values are real for every control value (A0 and every Ak
    // real there) come first: the kernels multiply them as real numbers.
    // The offset-0 band goes last: the kernels that fold it into the
    // own-entry coefficient then loop over the first nb - 1 bands only
    auto real_band = [&](int o) {
        auto is_real = [](const Bands &B, int o) {
            auto it = B.find(o);
            if (it == B.end()) return true;
            for (const cplx &c : it->second)
                if (c.imag() != 0.0) return false;
            return true;
        };
        if (!is_real(A0, o)) return false;
        for (const auto &B : Ak)
            if (!is_real(B, o)) return false;
        return true;
    };
    for (int pass = 0; pass < 2; ++pass)
        for (auto &kv : idx) {
            if (kv.first == 0 || real_band(kv.first) != (pass == 0)) continue;
            kv.second = (int)h.off.size();
            h.off.push_back(kv.first);
            if (pass == 0) h.nbr++;
        }
    if (idx.count(0)) {
        idx[0] = (int)h.off.size();
        h.off.push_back(0);
    }
    const int nb = (int)h.off.size(), R = (int)Ak.size();
    h.A0.assign((size_t)nb * d, cplx());
    h.Ak.assign((size_t)R * nb * d, cplx());
    for (const auto &kv : A0)
        for (int i = 0; i < d; ++i) h.A0[(size_t)idx[kv.first] * d + i] = kv.second[i];
    for (int k = 0; k < R; ++k)
        for (const auto &kv : Ak[k])
            for (int i = 0; i < d; ++i)
                h.Ak[((size_t)k * nb + idx[kv.first]) * d + i] = kv.second[i];
    for (size_t m = 0; m < jumps.size(); ++m)
        for (const auto &a : jumps[m])
            for (const auto &b : jumps[m]) {
                h.oL.push_back(a.first);
                h.oR.push_back(b.first);
                h.vL.insert(h.vL.end(), a.second.begin(), a.second.end());
                h.vR.insert(h.vR.end(), b.second.begin(), b.second.end());
                h.jctl.push_back(jump_ctl[m]);
            }
    return h;
}

// Where a caller's pointer lives, for a call on device `dev`: *on_dev is set
// for device memory of `dev` and for managed memory (the kernels read it
// directly), cleared for host memory (pageable, pinned or registered: it is
// copied through the problem's staging buffers).  Device memory of another
// device is rejected with GRAPE_EINVAL: the kernels would dereference peer
// memory, which faults without peer access.
grape_status locate_ptr(const void *p, int dev, const char *name, bool *on_dev) {
    *on_dev = false;
    if (!p) return GRAPE_OK;
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return GRAPE_OK;
    }
    if (a.type == cudaMemoryTypeManaged) {
        *on_dev = true;
    } else if (a.type == cudaMemoryTypeDevice) {
        if (a.device != dev)
            return fail(GRAPE_EINVAL, std::string(name) + " is device memory of device " +
                                          std::to_string(a.device) + ", not of the call's device " +
                                          std::to_string(dev));
        *on_dev = true;
    }
    return GRAPE_OK;
}

// locate_ptr for pointers that must be device memory of `dev`
grape_status require_device_ptr(const void *p, int dev, const char *name) {
    bool on_dev = false;
    const grape_status st = locate_ptr(p, dev, name, &on_dev);
    if (st != GRAPE_OK) return st;
    if (!on_dev) return fail(GRAPE_EINVAL, std::string(name) + " must be device memory");
    return GRAPE_OK;
}

int pow2ceil(long long x) {
    int p = 1;
    while (p < x) p <<= 1;
    return p;
}

class DeviceGuard {
  public:
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev_);
        if (prev_ != dev) cudaSetDevice(dev);
    }
    ~DeviceGuard() {
        int cur = -1;
        cudaGetDevice(&cur);
        if (cur != prev_) cudaSetDevice(prev_);
    }

  private:
    int prev_ = 0;
};

}  // namespace

struct grape_problem {
    int device = 0;
    int d = 0, R = 0, J = 0, ns = 0, n_slices = 0, n_rk = 0, mode = 0;
    int prec = GRAPE_PREC_DF64;      // number type of the kernels and of every state buffer
    double T = 0.0;
    size_t d2 = 0;
    int ncl = 1, threads = GRAPE_PROP_THREADS, chunk = 0, halo = 0, win = 0, reach = 0;
    int variant = 0;                 // bit 0 = real jump tables, bit 1 = Hermitian kernel
    int hb = 0, cu = 0, maxwin = 0, htab_len = 0, rt_rows = 0;   // Hermitian kernel geometry
    int fold = 0;                    // Hermitian kernel: own-entry coefficients cached in shared memory
    int jcache = 0;                  // Hermitian kernel: jump coefficients cached per entry
    int defer = 0;                   // Hermitian kernel: cluster wait after the compute
    int omax = 0;                    // largest band offset of either Lindbladian
    int hb_h = 0;                    // lower entries the Hermitian stencil reads
    std::map<int, int *> htabs;      // Hermitian tables per cluster width
    bool grid = false;               // grid kernel (state windows in global memory)
    int nblocks = 0;                 // its CTAs (n_states x ncl)
    unsigned *d_gflag = nullptr;     // its per-CTA round flags
    int *d_ntab = nullptr;           // its neighbour lists
    int ntab_stride = 0;
    long long spin_limit = 1LL << 22;   // grid-barrier polls (~0.3 s) before giving up
    double2 *d_gbuf = nullptr;
    unsigned *d_gbar = nullptr;
    int *d_htab = nullptr;
    size_t smem = 0;
    int ckpt_stride = 0;
    int seg = 0, nseg = 0;           // gradient segment plan (0 until first gradient)
    PropTables tab[2];               // [0] forward, [1] dual
    TraceArgs trace{};
    // state buffers hold 16-byte entries in the kernels' storage format
    // (double2 for FP64, float4 hi/lo pairs for double-float)
    double2 *d_rho0 = nullptr, *d_sigma = nullptr, *d_x = nullptr, *d_mu = nullptr;
    double2 *d_Y = nullptr, *d_K = nullptr, *d_ckpt = nullptr;
    double2 *d_out = nullptr;        // complex128 staging of rho(T)
    double *d_part = nullptr;        // per-split partial traces [n_slices][npairs][R]
    // filtered gradients: subpixel controls and their gradient [n_slices][R],
    // staged controls and gradient [n_steps][R] for host pointers
    double *d_fs = nullptr, *d_fgs = nullptr, *d_fu = nullptr, *d_fgu = nullptr;
    int f_steps = 0;
    // running-cost penalty (App. B): diagonal operator A, source -beta dt A,
    // per-boundary values Re Tr(A rho_n) summed over states [n_slices + 1],
    // boundary states of a chunked forward sweep
    bool penalty = false;
    double pen_beta = 0.0;
    double *d_pdiag = nullptr, *d_src = nullptr, *d_pen = nullptr;
    double2 *d_fwd_bounds = nullptr;
    static constexpr int kPenChunk = 64;
    double *d_u = nullptr, *d_F = nullptr, *d_G = nullptr;
    size_t bytes = 0;
    cudaStream_t s1 = nullptr;       // high-priority stream the gradient sweeps run on
    cudaStream_t s2 = nullptr;       // low-priority stream: traces overlap the adjoint sweep
    cudaStream_t s3 = nullptr;       // high-priority stream: the adjoint sweep beside the forward
    cudaEvent_t ev_fork = nullptr, ev_join = nullptr, ev_fork3 = nullptr;
    static constexpr int kMaxChunks = 16;
    cudaEvent_t ev[kMaxChunks + 2] = {};
    cudaEvent_t evF[kMaxChunks] = {};   // forward chunk c done (concurrent sweeps)
    bool profiling = false;
    struct Mark { int phase; cudaEvent_t a, b; };
    std::vector<Mark> marks;
    std::vector<cudaEvent_t> event_pool;
    cudaEvent_t take_event() {
        cudaEvent_t e = nullptr;
        if (!event_pool.empty()) {
            e = event_pool.back();
            event_pool.pop_back();
        } else if (cudaEventCreate(&e) != cudaSuccess) {
            cudaGetLastError();
            e = nullptr;
        }
        return e;
    }
    std::vector<void *> grad_allocs;   // gradient storage, released between served jobs
    size_t grad_bytes = 0;
    // Served jobs allocate gradient storage stream-ordered from the server's
    // pool (no device-wide synchronisation when a job starts or ends).
    cudaStream_t grad_stream = nullptr;
    cudaMemPool_t grad_pool = nullptr;
    void *alloc_grad(size_t n) {
        void *p = nullptr;
        const size_t nb = std::max<size_t>(n, 16);
        const cudaError_t e = grad_pool ? cudaMallocFromPoolAsync(&p, nb, grad_pool, grad_stream)
                                        : cudaMalloc(&p, nb);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        grad_allocs.push_back(p);
        grad_bytes += n;
        bytes += n;
        return p;
    }
    void release_grad() {
        for (void *p : grad_allocs) {
            if (grad_pool) cudaFreeAsync(p, grad_stream);
            else cudaFree(p);
        }
        grad_allocs.clear();
        grad_pool = nullptr;
        grad_stream = nullptr;
        bytes -= grad_bytes;
        grad_bytes = 0;
        d_Y = d_K = d_ckpt = nullptr;
        seg = nseg = 0;
    }
    std::vector<void *> allocs;
    void *alloc(size_t n) {
        void *p = nullptr;
        if (n == 0) n = 16;
        if (cudaMalloc(&p, n) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        allocs.push_back(p);
        bytes += n;
        return p;
    }
    ~grape_problem() {
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
        for (auto &e : evF)
            if (e) cudaEventDestroy(e);
        if (ev_fork3) cudaEventDestroy(ev_fork3);
        if (s3) cudaStreamDestroy(s3);
        if (s2) cudaStreamDestroy(s2);
        if (s1) cudaStreamDestroy(s1);
        if (ev_fork) cudaEventDestroy(ev_fork);
        if (ev_join) cudaEventDestroy(ev_join);
        if (!grad_pool)
            for (void *p : grad_allocs) cudaFree(p);
        for (auto &m : marks) { cudaEventDestroy(m.a); cudaEventDestroy(m.b); }
        for (auto e : event_pool) cudaEventDestroy(e);
        for (void *p : allocs) cudaFree(p);
    }
};

namespace {

template <typename T>
grape_status upload(grape_problem *P, const std::vector<T> &h, T **out) {
    *out = static_cast<T *>(P->alloc(h.size() * sizeof(T)));
    if (!*out) return fail(GRAPE_ENOMEM, "cudaMalloc failed for a problem table");
    if (!h.empty())
        GRAPE_CUDA_TRY(cudaMemcpy(*out, h.data(), h.size() * sizeof(T), cudaMemcpyHostToDevice));
    // a copy from pageable memory may return before its DMA lands, and the
    // kernels run on non-blocking streams that do not wait for the legacy
    // stream: wait for it here
    GRAPE_CUDA_TRY(cudaStreamSynchronize(cudaStreamLegacy));
    return GRAPE_OK;
}

double2 encode(const grape_problem *P, cplx v);

grape_status upload_dir(grape_problem *P, const HostDir &h, PropTables *t) {
    const int d = P->d;
    if ((int)h.off.size() > GRAPE_MAXB)
        return fail(GRAPE_EINVAL, "too many distinct Hamiltonian bands (max 12)");
    if ((int)h.oL.size() > GRAPE_MAXT)
        return fail(GRAPE_EINVAL, "too many jump band pairs (max 12)");
    std::memset(t, 0, sizeof(*t));
    t->nb = (int)h.off.size();
    t->nt = (int)h.oL.size();
    t->nbr = h.nbr;
    for (int b = 0; b < t->nb; ++b) {
        t->off[b] = h.off[b];
        t->off_row[b] = h.off[b] * d;
    }
    t->b0 = -1;
    for (int b = 0; b < t->nb; ++b)
        if (h.off[b] == 0) t->b0 = b;
    for (int q = 0; q < t->nt; ++q) {
        t->jflat[q] = h.oL[q] * d + h.oR[q];
        t->joL[q] = h.oL[q];
        t->joR[q] = h.oR[q];
        if (h.oL[q] == 0 && h.oR[q] == 0) t->jdiag |= 1 << q;
        t->jctl[q] = h.jctl[q];
        if (h.jctl[q] >= 0) t->jrate |= 1 << q;
    }
    auto cvt = [](const std::vector<cplx> &v) {
        std::vector<double2> o(v.size());
        for (size_t i = 0; i < v.size(); ++i) o[i] = make_double2(v[i].real(), v[i].imag());
        return o;
    };
    double2 *p;
    grape_status s;
    if ((s = upload(P, cvt(h.vL), &p)) != GRAPE_OK) return s;
    t->vL = p;
    if ((s = upload(P, cvt(h.vR), &p)) != GRAPE_OK) return s;
    t->vR = p;
    auto enc = [&](const std::vector<cplx> &v) {
        std::vector<double2> o(v.size());
        for (size_t i = 0; i < v.size(); ++i) o[i] = encode(P, v[i]);
        return o;
    };
    if ((s = upload(P, enc(h.A0), &p)) != GRAPE_OK) return s;
    t->A0s = p;
    if ((s = upload(P, enc(h.Ak), &p)) != GRAPE_OK) return s;
    t->Aks = p;
    if ((s = upload(P, enc(h.vL), &p)) != GRAPE_OK) return s;
    t->vLs = p;
    if ((s = upload(P, enc(h.vR), &p)) != GRAPE_OK) return s;
    t->vRs = p;
    return GRAPE_OK;
}

// Kernel launches in the problem's number type.
cudaError_t k_prop(const grape_problem *P, const PropArgs &a, cudaStream_t s) {
    if (P->grid) {
        // arrivals and generation restart at zero; the error flag is kept
        // until grape_problem_status reads it
        // round flags restart at zero; the error word is kept until
        // grape_problem_status reads it
        const cudaError_t e = cudaMemsetAsync(P->d_gflag, 0, (size_t)P->nblocks * sizeof(unsigned), s);
        if (e != cudaSuccess) return e;
        return P->prec == GRAPE_PREC_FP64 ? grape_launch_grid_f64(a, P->nblocks, P->variant, P->smem, s)
                                          : grape_launch_grid_df(a, P->nblocks, P->variant, P->smem, s);
    }
    return P->prec == GRAPE_PREC_FP64 ? grape_launch_prop_f64(a, P->threads, P->variant, P->smem, s)
                                      : grape_launch_prop_df(a, P->threads, P->variant, P->smem, s);
}
cudaError_t k_trace(const grape_problem *P, const TraceArgs &t, cudaStream_t s) {
    return P->prec == GRAPE_PREC_FP64 ? grape_launch_trace_f64(t, s) : grape_launch_trace_df(t, s);
}
cudaError_t k_cost(const grape_problem *P, const void *rho, double *F, cudaStream_t s) {
    return P->prec == GRAPE_PREC_FP64
               ? grape_launch_cost_f64(rho, P->d_sigma, P->ns, (int)P->d2, F, s)
               : grape_launch_cost_df(rho, P->d_sigma, P->ns, (int)P->d2, F, s);
}
cudaError_t k_to_double(const grape_problem *P, const void *src, double2 *dst, size_t n,
                        cudaStream_t s) {
    return P->prec == GRAPE_PREC_FP64 ? grape_launch_to_double_f64(src, dst, n, s)
                                      : grape_launch_to_double_df(src, dst, n, s);
}

// complex128 -> one 16-byte storage entry
double2 encode(const grape_problem *P, cplx v) {
    if (P->prec == GRAPE_PREC_FP64) return make_double2(v.real(), v.imag());
    const grape_num::ff re = grape_num::ff_from_double(v.real());
    const grape_num::ff im = grape_num::ff_from_double(v.imag());
    const float4 f = make_float4(re.h, im.h, re.l, im.l);   // the kernels' pair layout
    double2 out;
    std::memcpy(&out, &f, sizeof(out));
    return out;
}

int max_smem_optin(const grape_problem *P) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, P->device) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return v;
}

// True when at least one cluster of `ncl` CTAs of `threads` threads and
// `smem` bytes of dynamic shared memory can be resident.
bool cluster_fits(const grape_problem *P, int variant, int threads, size_t smem, int ncl) {
    int clusters = 0;
    const cudaError_t e =
        P->prec == GRAPE_PREC_FP64
            ? grape_max_active_clusters_f64(threads, variant, smem, ncl, ncl * P->ns, &clusters)
            : grape_max_active_clusters_df(threads, variant, smem, ncl, ncl * P->ns, &clusters);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return clusters >= 1;
}

// Full-matrix cluster kernel with `ncl` CTAs of `threads` threads per state:
// sets the geometry, or GRAPE_EINVAL when the tile does not fit.
grape_status plan_full(grape_problem *P, int ncl, int threads) {
    const int max_smem = max_smem_optin(P);
    const long long d2 = (long long)P->d2;
    const int halo = P->omax * (P->d + 1);
    const int nb = std::max(P->tab[0].nb, P->tab[1].nb), nt = std::max(P->tab[0].nt, P->tab[1].nt);
    const int chunk = (int)((d2 + ncl - 1) / ncl);
    const int win = chunk + 2 * halo;
    // windows, base values and accumulators, bands, jump tables (16 B each),
    // the (row, column) table of the owned entries and 12 RK coefficients
    const size_t smem = ((size_t)2 * win + 2 * (size_t)chunk + 2 * (size_t)nb * P->d +
                         2 * (size_t)nt * P->d) * sizeof(double2) +
                        (size_t)chunk * sizeof(int2) + 12 * sizeof(double);
    const int variant = P->variant & 1;
    if (smem + 1024 > (size_t)max_smem)   // keep room for static shared memory
        return fail(GRAPE_EINVAL, "state window does not fit in shared memory");
    if (!cluster_fits(P, variant, threads, smem, ncl))
        return fail(GRAPE_EINVAL, "no cluster of this shape can be resident");
    P->variant = variant;
    P->ncl = ncl;
    P->halo = halo;
    P->chunk = chunk;
    P->win = win;
    P->smem = smem;
    P->threads = threads;
    P->reach = (ncl > 1) ? (halo + chunk - 1) / chunk : 0;
    return GRAPE_OK;
}

// Preferred width first, then wider, then narrower (bounded search).
int candidate_widths(int start, int *widths) {
    int nw = 0;
    for (int c = start; c <= 16; c *= 2) widths[nw++] = c;
    for (int c = start / 2; c >= 1; c /= 2) widths[nw++] = c;
    return nw;
}

int env_cluster(int start) {
    if (const char *env = std::getenv("GRAPE_CLUSTER")) {
        const int v = std::atoi(env);
        if (v == 1 || v == 2 || v == 4 || v == 8 || v == 16) return v;
    }
    return start;
}

grape_status choose_geometry(grape_problem *P) {
    const long long d2 = (long long)P->d2;
    const int start = env_cluster(std::min(16, pow2ceil((d2 + 1023) / 1024)));
    cudaError_t e = P->prec == GRAPE_PREC_FP64
                        ? grape_prepare_prop_f64(P->variant & 1, (size_t)max_smem_optin(P), 16)
                        : grape_prepare_prop_df(P->variant & 1, (size_t)max_smem_optin(P), 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(GRAPE_ECUDA, std::string("prop kernel attributes: ") + cudaGetErrorString(e));
    }
    int widths[8];
    const int nw = candidate_widths(start, widths);
    for (int wi = 0; wi < nw; ++wi)
        if (plan_full(P, widths[wi], GRAPE_PROP_THREADS) == GRAPE_OK) return GRAPE_OK;
    return fail(GRAPE_EINVAL, "problem too large for the cluster propagation kernel "
                              "(state window does not fit in shared memory)");
}

// Geometry of the Hermitian (upper-triangle) kernel for a cluster of ncl
// CTAs: ownership ranges, compact windows and the table described in
// grape_internal.h.  Returns the table, the largest window and the entries
// per CTA.
std::vector<int> hermitian_table(int d, int ncl, int omax, int hb, int *maxwin, int *cu,
                                 int *rt_rows) {
    const long long NU = (long long)d * (d + 1) / 2;
    const int c = (int)((NU + ncl - 1) / ncl);
    auto row_start = [d](long long i) { return i * d - i * (i - 1) / 2; };
    auto row_of = [&](long long u) {
        long long lo = 0, hi = d - 1;
        while (lo < hi) {
            const long long mid = (lo + hi + 1) / 2;
            if (row_start(mid) <= u) lo = mid; else hi = mid - 1;
        }
        return (int)lo;
    };
    auto cs = [hb](int r) { return r > hb ? r - hb : 0; };
    std::vector<int> head(4 * ncl), starts(ncl + 1), lists;
    std::vector<int> wr0(ncl), wr1(ncl);
    int mw = 0, rt = 1;
    for (int k = 0; k < ncl; ++k) {
        const long long u0 = std::min<long long>(NU, (long long)k * c);
        const long long u1 = std::min<long long>(NU, u0 + c);
        int r0 = 0, nrows = 0;
        if (u1 > u0) {
            // rows written by the CTA: its own and, for mirrors, hb below
            rt = std::max(rt, std::min(d - 1, row_of(u1 - 1) + hb) - row_of(u0) + 1);
            r0 = std::max(0, row_of(u0) - omax);
            const int r1 = std::min(d - 1, row_of(u1 - 1) + omax);
            nrows = r1 - r0 + 1;
        }
        head[4 * k + 0] = (int)u0;
        head[4 * k + 1] = (int)u1;
        head[4 * k + 2] = r0;
        head[4 * k + 3] = nrows;
        wr0[k] = r0;
        wr1[k] = r0 + nrows - 1;
        starts[k] = 4 * ncl + ncl + 1 + (int)lists.size();
        int acc = 0;
        lists.push_back(0);
        for (int r = r0; r < r0 + nrows; ++r) {
            acc += d - cs(r);
            lists.push_back(acc);
        }
        mw = std::max(mw, acc);
    }
    starts[ncl] = 4 * ncl + ncl + 1 + (int)lists.size();
    std::vector<int> kf(d, ncl), kl(d, -1);
    for (int k = 0; k < ncl; ++k)
        for (int r = wr0[k]; r <= wr1[k]; ++r) {
            kf[r] = std::min(kf[r], k);
            kl[r] = std::max(kl[r], k);
        }
    std::vector<int> tab;
    tab.insert(tab.end(), head.begin(), head.end());
    tab.insert(tab.end(), starts.begin(), starts.end());
    tab.insert(tab.end(), lists.begin(), lists.end());
    tab.insert(tab.end(), kf.begin(), kf.end());
    tab.insert(tab.end(), kl.begin(), kl.end());
    *maxwin = mw;
    *cu = c;
    *rt_rows = rt;
    return tab;
}

// The compile-time band/jump layout (the kernels' Shape) that both
// directions' tables follow: 1 transmon x resonator (bands 0, +-1 real,
// +-Q; three jump terms), 2 resonator drives only (bands 0, +-Q; one jump
// term), 0 none (the kernels read the counts at run time).  Real jump tables
// only; GRAPE_SHAPE=0 turns it off.  The arithmetic is the same either way.
int shape_id(const grape_problem *P) {
    if (!(P->variant & 1)) return 0;
    if (const char *env = std::getenv("GRAPE_SHAPE"))
        if (std::atoi(env) == 0) return 0;
    auto is = [&](int nb, int nbr, int nt) {
        for (int dir = 0; dir < 2; ++dir) {
            const PropTables &t = P->tab[dir];
            if (t.nb != nb || t.nbr != nbr || t.nt != nt || t.b0 != nb - 1) return false;
        }
        return true;
    };
    if (is(5, 2, 3)) return 1;
    if (is(3, 0, 1)) return 2;
    return 0;
}

// Hermitian cluster kernel with `ncl` CTAs of `threads` threads per state:
// sets the geometry, or GRAPE_EINVAL when the tile does not fit.  Tables
// are kept per width (a captured graph may still use an earlier one).
grape_status plan_h(grape_problem *P, int ncl, int threads) {
    const int max_smem = max_smem_optin(P);
    const int d = P->d, hb = P->hb_h;
    const int nb = std::max(P->tab[0].nb, P->tab[1].nb), nt = std::max(P->tab[0].nt, P->tab[1].nt);
    int maxwin = 0, cu = 0, rt_rows = 0;
    const std::vector<int> tab = hermitian_table(d, ncl, P->omax, hb, &maxwin, &cu, &rt_rows);
    if (maxwin >= 32767) return fail(GRAPE_EINVAL, "state window too large for 16-bit addresses");
    // shared memory without windows, own-entry and jump-coefficient tables
    // two mbarriers; base values, accumulators and next values of the owned
    // entries; bands, jump tables; (row, column), RK coefficients, the
    // window table, the row push table (address and mbarrier per target)
    // and the neighbour addresses
    const size_t base = 16 + (2 * (size_t)cu + 2 * (size_t)nb * d + 2 * (size_t)nt * d) * sizeof(double2) +
                        (size_t)cu * sizeof(int2) + 12 * sizeof(double) + tab.size() * sizeof(int) +
                        (size_t)rt_rows * (2 * ncl + 1) * sizeof(uint32_t) +
                        (size_t)cu * (2 * nb + nt + 1) * sizeof(short);
    const int sh = shape_id(P);
    const int variant = (P->variant & 1) | 2 | (sh << 2) | ((sh && cu <= threads) ? 16 : 0);
    {
        const cudaError_t e = P->prec == GRAPE_PREC_FP64
                                  ? grape_prepare_prop_f64(variant, (size_t)max_smem_optin(P), 16)
                                  : grape_prepare_prop_df(variant, (size_t)max_smem_optin(P), 16);
        if (e != cudaSuccess) {
            cudaGetLastError();
            return fail(GRAPE_ECUDA, std::string("hermitian kernel attributes: ") + cudaGetErrorString(e));
        }
    }
    // Options, each kept only when the tile still fits (the same values, so
    // the same bits, either way): the own-entry coefficients cached per slice
    // (16 B per owned entry) instead of recomputed every stage; the next
    // values of the owned entries kept in a row (16 B per owned entry) so
    // that the cluster wait before the pushes comes after the compute; the
    // jump coefficients of real jump tables cached per entry (8 B per term
    // with an offset and owned entry).
    bool want_fold = true, want_defer = false, want_jc = (variant & 1) != 0;
    if (const char *env = std::getenv("GRAPE_FOLD")) want_fold = std::atoi(env) != 0;
    if (const char *env = std::getenv("GRAPE_DEFER")) want_defer = std::atoi(env) != 0;   // off: measured slower
    if (variant & 16) want_defer = false;        // one entry per thread: the wait stays before the compute
    if (const char *env = std::getenv("GRAPE_JCACHE")) want_jc = want_jc && std::atoi(env) != 0;
    int njt = 0;
    for (int q = 0; q < P->tab[0].nt; ++q) njt += ((P->tab[0].jdiag >> q) & 1) ? 0 : 1;
    int njt_d = 0;
    for (int q = 0; q < P->tab[1].nt; ++q) njt_d += ((P->tab[1].jdiag >> q) & 1) ? 0 : 1;
    njt = std::max(njt, njt_d);
    struct Opt { bool fold, defer, jc; };
    const Opt opts[] = {{true, true, true}, {true, true, false}, {true, false, true}, {true, false, false},
                        {false, true, false}, {false, false, false}};
    size_t use = 0;
    bool found = false, fold = false, defer = false, jcache = false;
    for (const Opt &o : opts) {
        if ((o.fold && !want_fold) || (o.defer && !want_defer) || (o.jc && !want_jc)) continue;
        const size_t sm = base + 2 * (size_t)(maxwin + 1) * sizeof(double2) +
                          (o.fold ? (size_t)cu * sizeof(double2) : 0) +
                          (o.defer ? (size_t)cu * sizeof(double2) : 0) +
                          (o.jc ? (size_t)njt * cu * sizeof(double) : 0);
        if (sm + 1024 > (size_t)max_smem || !cluster_fits(P, variant, threads, sm, ncl)) continue;
        use = sm;
        fold = o.fold;
        defer = o.defer;
        jcache = o.jc;
        found = true;
        break;
    }
    if (!found) {
        const size_t least = base + 2 * (size_t)(maxwin + 1) * sizeof(double2);
        if (least + 1024 > (size_t)max_smem) return fail(GRAPE_EINVAL, "state window does not fit in shared memory");
        return fail(GRAPE_EINVAL, "no cluster of this shape can be resident");
    }
    auto it = P->htabs.find(ncl);
    if (it == P->htabs.end()) {
        int *dt = nullptr;
        grape_status st = upload(P, tab, &dt);
        if (st != GRAPE_OK) return st;
        it = P->htabs.emplace(ncl, dt).first;
    }
    P->d_htab = it->second;
    P->variant = variant;
    P->ncl = ncl;
    P->cu = cu;
    P->maxwin = maxwin;
    P->hb = hb;
    P->htab_len = (int)tab.size();
    P->rt_rows = rt_rows;
    P->smem = use;
    P->fold = fold ? 1 : 0;

    P->jcache = jcache ? 1 : 0;
    P->defer = defer ? 1 : 0;
    P->threads = threads;
    P->chunk = cu;
    P->halo = 0;
    P->win = maxwin;
    P->reach = 0;
    return GRAPE_OK;
}

grape_status choose_geometry_h(grape_problem *P) {
    const long long NU = (long long)P->d * (P->d + 1) / 2;
    const int start = env_cluster(std::min(16, pow2ceil((NU + 511) / 512)));
    const int variant = (P->variant & 1) | 2;
    cudaError_t e = P->prec == GRAPE_PREC_FP64 ? grape_prepare_prop_f64(variant, (size_t)max_smem_optin(P), 16)
                                               : grape_prepare_prop_df(variant, (size_t)max_smem_optin(P), 16);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return fail(GRAPE_ECUDA, std::string("hermitian kernel attributes: ") + cudaGetErrorString(e));
    }
    int widths[8];
    const int nw = candidate_widths(start, widths);
    for (int wi = 0; wi < nw; ++wi) {
        const grape_status st = plan_h(P, widths[wi], GRAPE_PROP_THREADS);
        if (st == GRAPE_OK && P->ncl == 1) {
            // one CTA per state: whole warps for the owned entries only, so
            // the per-stage CTA barrier waits on fewer warps (d=20: 4.15
            // against 4.38 ms per gradient with 512 threads, same bits)
            const int t = std::max(64, (P->cu + 31) / 32 * 32);
            if (t < GRAPE_PROP_THREADS && plan_h(P, 1, t) != GRAPE_OK) return plan_h(P, 1, GRAPE_PROP_THREADS);
        }
        if (st == GRAPE_OK || st != GRAPE_EINVAL) return st;
    }
    return fail(GRAPE_EINVAL, "problem too large for the Hermitian cluster kernel");
}

// Neighbour lists of the grid kernel's CTAs (of one state): a and b are
// neighbours when one writes a row the other's window holds.  The rows a
// CTA writes lie in [first own row, last own row + hb] (its own rows and
// the mirror rows of its entries near the diagonal).  Row k of the table:
// the count, then the ranks; *stride = 1 + the largest count.
std::vector<int> neighbour_table(const std::vector<int> &tab, int d, int nct, int hb, int *stride) {
    auto row_start = [d](long long i) { return i * d - i * (i - 1) / 2; };
    auto row_of = [&](long long u) {
        long long lo = 0, hi = d - 1;
        while (lo < hi) {
            const long long mid = (lo + hi + 1) / 2;
            if (row_start(mid) <= u) lo = mid; else hi = mid - 1;
        }
        return (int)lo;
    };
    std::vector<int> r0(nct, 1), r1(nct, 0), w0(nct), w1(nct);
    for (int k = 0; k < nct; ++k) {
        const long long u0 = tab[GRAPE_HTAB_CTA(k) + 0], u1 = tab[GRAPE_HTAB_CTA(k) + 1];
        if (u1 > u0) {
            r0[k] = row_of(u0);
            r1[k] = std::min(d - 1, row_of(u1 - 1) + hb);
        }
        w0[k] = tab[GRAPE_HTAB_CTA(k) + 2];
        w1[k] = w0[k] + tab[GRAPE_HTAB_CTA(k) + 3] - 1;
    }
    auto writes_into = [&](int a, int b) { return r0[a] <= r1[a] && w0[b] <= w1[b] && r0[a] <= w1[b] && w0[b] <= r1[a]; };
    std::vector<std::vector<int>> nbrs(nct);
    size_t mx = 0;
    for (int a = 0; a < nct; ++a) {
        for (int b = 0; b < nct; ++b)
            if (a != b && (writes_into(a, b) || writes_into(b, a))) nbrs[a].push_back(b);
        mx = std::max(mx, nbrs[a].size());
    }
    *stride = (int)mx + 1;
    std::vector<int> out((size_t)nct * *stride, 0);
    for (int a = 0; a < nct; ++a) {
        out[(size_t)a * *stride] = (int)nbrs[a].size();
        for (size_t t = 0; t < nbrs[a].size(); ++t) out[(size_t)a * *stride + 1 + t] = nbrs[a][t];
    }
    return out;
}

// Grid kernel: nct CTAs per state, one per SM (all resident), the
// Hermitian kernel's ownership and window tables over nct CTAs.
grape_status choose_geometry_grid(grape_problem *P) {
    int max_smem = 0, sms = 0;
    GRAPE_CUDA_TRY(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, P->device));
    GRAPE_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, P->device));
    const int d = P->d, hb = P->hb_h;
    const int nb = std::max(P->tab[0].nb, P->tab[1].nb), nt = std::max(P->tab[0].nt, P->tab[1].nt);
    int nct = std::max(1, sms / P->ns);
    if (const char *env = std::getenv("GRAPE_GRID_BLOCKS")) {
        const long long v = std::atoll(env);
        if (v > 0) nct = (int)std::max<long long>(1, std::min<long long>(v / P->ns, sms / P->ns));
    }
    int maxwin = 0, cu = 0, rt_rows = 0;
    const std::vector<int> tab = hermitian_table(d, nct, P->omax, hb, &maxwin, &cu, &rt_rows);
    if (maxwin >= 32767) return fail(GRAPE_EINVAL, "state window too large for the grid propagation kernel");
    const int variant = (P->variant & 1) | (shape_id(P) << 2);
    int njt = 0;
    for (int dir = 0; dir < 2; ++dir) {
        int n = 0;
        for (int q = 0; q < P->tab[dir].nt; ++q) n += ((P->tab[dir].jdiag >> q) & 1) ? 0 : 1;
        njt = std::max(njt, n);
    }
    // one window, base values and accumulators, one band table (the jump
    // tables stay in global memory)
    const size_t base = ((size_t)(maxwin + 1) + 2 * (size_t)cu + (size_t)nb * d) * sizeof(double2) +
                        (size_t)cu * sizeof(int2) + 12 * sizeof(double) + tab.size() * sizeof(int) +
                        (size_t)cu * (2 * nb + nt + 1) * sizeof(short);
    bool want_fold = true, want_jc = variant != 0;
    if (const char *env = std::getenv("GRAPE_FOLD")) want_fold = std::atoi(env) != 0;
    if (const char *env = std::getenv("GRAPE_JCACHE")) want_jc = want_jc && std::atoi(env) != 0;
    struct Opt { bool fold, jc; };
    const Opt opts[] = {{true, true}, {true, false}, {false, true}, {false, false}};
    size_t smem = 0;
    bool found = false, fold = false, jcache = false;
    for (const Opt &o : opts) {
        if ((o.fold && !want_fold) || (o.jc && !want_jc)) continue;
        const size_t sm = base + (o.fold ? (size_t)cu * sizeof(double2) : 0) +
                          (o.jc ? (size_t)njt * cu * sizeof(double) : 0);
        if (sm + 1024 > (size_t)max_smem) continue;
        int max_blocks = 0;
        const cudaError_t e = P->prec == GRAPE_PREC_FP64
                                  ? grape_prepare_grid_f64(variant, (size_t)max_smem, sm, &max_blocks)
                                  : grape_prepare_grid_df(variant, (size_t)max_smem, sm, &max_blocks);
        if (e != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (max_blocks < nct * P->ns) continue;   // every CTA must be resident
        smem = sm;
        fold = o.fold;
        jcache = o.jc;
        found = true;
        break;
    }
    if (!found) return fail(GRAPE_EINVAL, "problem too large for the grid propagation kernel");
    int stride = 0;
    const std::vector<int> ntab = neighbour_table(tab, d, nct, hb, &stride);
    grape_status st;
    if ((st = upload(P, tab, &P->d_htab)) != GRAPE_OK) return st;
    if ((st = upload(P, ntab, &P->d_ntab)) != GRAPE_OK) return st;
    P->d_gbuf = static_cast<double2 *>(P->alloc((size_t)2 * P->ns * P->d2 * sizeof(double2)));
    P->d_gflag = static_cast<unsigned *>(P->alloc((size_t)nct * P->ns * sizeof(unsigned)));
    if (!P->d_gbuf || !P->d_gflag) return fail(GRAPE_ENOMEM, "cudaMalloc failed for the grid kernel buffers");
    if (const char *env = std::getenv("GRAPE_SPIN_LIMIT")) P->spin_limit = std::atoll(env);
    P->grid = true;
    P->variant = variant;
    P->nblocks = nct * P->ns;
    P->ncl = nct;
    P->cu = cu;
    P->maxwin = maxwin;
    P->hb = hb;
    P->htab_len = (int)tab.size();
    P->rt_rows = rt_rows;
    P->fold = fold ? 1 : 0;
    P->jcache = jcache ? 1 : 0;
    P->ntab_stride = stride;
    P->smem = smem;
    P->threads = GRAPE_GRID_THREADS;
    P->chunk = cu;
    return GRAPE_OK;
}

void rk_coefficients(double h, bool adjoint, PropArgs *a) {
    if (!adjoint) {
        const double g[4] = {1.0, 1.0, 1.0, 1.0};
        const double w[4] = {h / 6, h / 3, h / 3, h / 6};
        const double b[4] = {0.0, h / 2, h / 2, h};
        for (int s = 0; s < 4; ++s) { a->g[s] = g[s]; a->a[s] = w[s]; a->b[s] = b[s]; a->store_map[s] = s; }
    } else {
        // reverse mode of one RK4 substep: kb4 = h/6 mu, kb3 = h/3 mu + h yb4,
        // kb2 = h/3 mu + h/2 yb3, kb1 = h/6 mu + h/2 yb2; mu_prev = mu + sum yb
        const double g[4] = {h / 6, h / 3, h / 3, h / 6};
        const double b[4] = {0.0, h, h / 2, h / 2};
        for (int s = 0; s < 4; ++s) { a->g[s] = g[s]; a->a[s] = 1.0; a->b[s] = b[s]; a->store_map[s] = 3 - s; }
    }
}

PropArgs base_args(const grape_problem *P, int dir, const double *u) {
    PropArgs a;
    std::memset(&a, 0, sizeof(a));
    a.tab = P->tab[dir];
    a.d = P->d;
    a.R = P->R;
    a.n_states = P->ns;
    a.ncl = P->ncl;
    a.chunk = P->chunk;
    a.halo = P->halo;
    a.win = P->win;
    a.reach = P->reach;
    a.u = u;
    a.n_rk = P->n_rk;
    a.bound_step = 1;
    a.htab = P->d_htab;
    a.htab_len = P->htab_len;
    a.hb = P->hb;
    a.cu = P->cu;
    a.maxwin = P->maxwin;
    a.rt_rows = P->rt_rows;
    a.fold = ((P->variant & 2) || P->grid) ? P->fold : 0;

    a.jcache = ((P->variant & 2) || P->grid) ? P->jcache : 0;
    a.defer = (P->variant & 2) ? P->defer : 0;
    a.src = P->penalty ? P->d_src : nullptr;
    a.gbuf = P->d_gbuf;
    a.gbar = P->d_gbar;
    a.gflag = P->d_gflag;
    a.ntab = P->d_ntab;
    a.ntab_stride = P->ntab_stride;
    a.spin_limit = P->spin_limit;
    rk_coefficients(P->T / P->n_slices / P->n_rk, dir == 1, &a);
    return a;
}

// Entries of one set of stored stage values (all states): the exact
// gradient's stage storage holds packed upper triangles (d(d+1)/2 entries
// per state), the first-order mode's slice boundaries and the checkpoints
// hold full matrices (d^2).
size_t packed_set(const grape_problem *P) { return (size_t)P->d * (P->d + 1) / 2 * P->ns; }
size_t full_set(const grape_problem *P) { return P->d2 * P->ns; }

// stage storage of one segment, Y or K, in bytes
size_t stage_bytes(const grape_problem *P, long long seg) {
    return (P->mode == GRAPE_GRAD_EXACT) ? (size_t)seg * P->n_rk * 4 * packed_set(P) * sizeof(double2)
                                         : (size_t)(seg + 1) * full_set(P) * sizeof(double2);
}
// checkpoints of a segment plan, in bytes
size_t ckpt_bytes(const grape_problem *P, long long seg) {
    return seg < P->n_slices ? (size_t)((P->n_slices + seg - 1) / seg + 1) * full_set(P) * sizeof(double2) : 0;
}

size_t seg_bytes(const grape_problem *P, long long seg) {
    return 2 * stage_bytes(P, seg) + ckpt_bytes(P, seg);
}

// Device buffers one gradient evaluation needs beyond its inputs and outputs.
struct GradScratch {
    double2 *Y = nullptr, *K = nullptr, *ckpt = nullptr, *x = nullptr, *mu = nullptr;
    int seg = 0, nseg = 0;
    cudaStream_t s2 = nullptr;   // trace stream; null: traces run on the main stream
    cudaEvent_t *ev = nullptr;   // kMaxChunks + 2 events when s2 is set
    double *part = nullptr;      // partial traces; null: one CTA per slice
    // concurrent sweeps (see concurrent_sweeps): the adjoint's stream, its
    // fork event and the forward chunks' events; null: one sweep after the other
    cudaStream_t s3 = nullptr;
    cudaEvent_t fork3 = nullptr;
    cudaEvent_t *evF = nullptr;
};

long long trace_pairs(const grape_problem *P) {
    return (P->mode == GRAPE_GRAD_EXACT) ? (long long)P->n_rk * 4 * P->ns : (long long)P->ns;
}

// Splits of each slice's trace over CTAs, constants of the problem (so the
// summation order, and with it every bit of the gradient, does not depend on
// how the slices are grouped into launches or on the propagation tile).
// Exact gradient (packed storage): per state, chunks of 256 x epc upper
// entries, epc chosen so that a state has at most 64 chunks.  First-order
// mode (full matrices): contiguous ranges of the slice's pairs worth about
// 2^17 band-element products each.
void trace_layout(const grape_problem *P, TraceArgs *t) {
    t->n_states = P->ns;
    if (P->mode == GRAPE_GRAD_EXACT) {
        const long long nu = (long long)P->d * (P->d + 1) / 2;
        t->packed = 1;
        t->epc = (int)std::max<long long>(1, (nu + 256 * 64 - 1) / (256 * 64));
        t->nchunk = (int)((nu + 256LL * t->epc - 1) / (256LL * t->epc));
        t->nsplit = P->ns * t->nchunk;
        return;
    }
    const long long npairs = trace_pairs(P);
    const long long work = (long long)P->d * P->d * std::max(1, t->ndo);
    const long long per = std::max<long long>(1, ((1LL << 17) + work - 1) / work);
    t->packed = 0;
    t->epc = t->nchunk = 1;
    t->nsplit = (int)std::max<long long>(1, (npairs + per - 1) / per);
}

// Tables of the packed trace kernels: the row and column of every packed
// entry, and for the staged kernel (no rate-controlled dissipators, at most 4
// distinct control offsets): per 256-entry block of
// the packed triangle, the runs of packed K positions its entries'
// neighbours (i+o, j) and (i, j+o) fall in (gaps of up to 8 entries are
// copied along, so one run can span the end of a row and the start of the
// next), and per entry the neighbours' indices in the block's K buffer.
// Left off (the fast kernel runs) when GRAPE_TRACE=fast or the buffers do
// not fit shared memory.
grape_status trace_tiles(grape_problem *P, TraceArgs *t) {
    t->err = P->d_gbar + 2;
    t->tile = 0;
    // bound of the staged kernel's copy waits: about a second of SM clocks;
    // GRAPE_TRACE_SPIN=n overrides it (0: every wait gives up at once, the
    // error path; the copies already issued are still waited for)
    t->spin = 1LL << 31;
    if (const char *env = std::getenv("GRAPE_TRACE_SPIN")) t->spin = std::max(0LL, std::atoll(env));
    if (!t->packed) return GRAPE_OK;
    const int d = P->d;
    if (d > 65535) return fail(GRAPE_EINVAL, "d above 65535 (16-bit row and column indices)");
    const long long NU = (long long)d * (d + 1) / 2;
    // row and column of every packed entry (all packed trace kernels)
    std::vector<unsigned> ij((size_t)NU);
    {
        size_t u = 0;
        for (int i = 0; i < d; ++i)
            for (int j = i; j < d; ++j) ij[u++] = (unsigned)i | ((unsigned)j << 16);
    }
    {
        unsigned *dij = nullptr;
        const grape_status st = upload(P, ij, &dij);
        if (st != GRAPE_OK) return st;
        t->tij = dij;
    }
    if (t->nst != 0 || t->ndo <= 0 || t->ndo > 4) return GRAPE_OK;
    if (const char *env = std::getenv("GRAPE_TRACE"))
        if (std::string(env) == "fast") return GRAPE_OK;
    auto pk = [d](long long r, long long c) { return r * d - r * (r - 1) / 2 + (c - r); };
    const long long nblk = (NU + 255) / 256;
    std::vector<int4> blk((size_t)nblk), runs;
    std::vector<uint4> nb((size_t)NU);
    std::vector<long long> pos;
    std::vector<long long> rs, rl, ro;                       // the block's runs: start, length, offset
    int kcap = 0;
    for (long long b = 0; b < nblk; ++b) {
        const long long u0 = b * 256, u1 = std::min(NU, u0 + 256);
        // stored position of neighbour `which` (0: (i+o, j), 1: (i, j+o)) of
        // entry u at offset index oi, -1 when outside; *cj: the mirror is stored
        auto nbpos = [&](long long u, int oi, int which, bool *cj) -> long long {
            const int i = (int)(ij[u] & 0xffffu), j = (int)(ij[u] >> 16);
            const int o = t->do_off[oi];
            *cj = false;
            if (which == 0) {
                const int r1 = i + o;
                if (r1 < 0 || r1 >= d) return -1;
                *cj = r1 > j;
                return *cj ? pk(j, r1) : pk(r1, j);
            }
            const int c2 = j + o;
            if (i >= j || c2 < 0 || c2 >= d) return -1;
            *cj = c2 < i;
            return *cj ? pk(c2, i) : pk(i, c2);
        };
        pos.clear();
        for (long long u = u0; u < u1; ++u)
            for (int oi = 0; oi < t->ndo; ++oi)
                for (int w = 0; w < 2; ++w) {
                    bool cj;
                    const long long x = nbpos(u, oi, w, &cj);
                    if (x >= 0) pos.push_back(x);
                }
        std::sort(pos.begin(), pos.end());
        pos.erase(std::unique(pos.begin(), pos.end()), pos.end());
        rs.clear();
        rl.clear();
        ro.clear();
        long long klen = 0;
        for (long long x : pos) {
            if (!rs.empty() && x - (rs.back() + rl.back()) <= 8) {
                klen += x + 1 - (rs.back() + rl.back());
                rl.back() = x - rs.back() + 1;
            } else {
                rs.push_back(x);
                rl.push_back(1);
                ro.push_back(klen);
                klen += 1;
            }
        }
        if (klen > 32767) return GRAPE_OK;                    // 15-bit buffer indices
        kcap = std::max(kcap, (int)klen);
        blk[(size_t)b] = make_int4((int)runs.size(), (int)rs.size(), (int)klen, 0);
        for (size_t r = 0; r < rs.size(); ++r) runs.push_back(make_int4((int)rs[r], (int)rl[r], (int)ro[r], 0));
        for (long long u = u0; u < u1; ++u) {
            unsigned w16[8];
            for (int k = 0; k < 8; ++k) {
                w16[k] = 0xffffu;
                const int oi = k >> 1;
                if (oi >= t->ndo) continue;
                bool cj;
                const long long x = nbpos(u, oi, k & 1, &cj);
                if (x < 0) continue;
                const size_t r = (size_t)(std::upper_bound(rs.begin(), rs.end(), x) - rs.begin()) - 1;
                w16[k] = (unsigned)(ro[r] + (x - rs[r])) | (cj ? 0x8000u : 0u);
            }
            nb[(size_t)u] = make_uint4(w16[0] | w16[1] << 16, w16[2] | w16[3] << 16, w16[4] | w16[5] << 16,
                                       w16[6] | w16[7] << 16);
        }
    }
    // buffers: as many (2 to 4) as fit 104 KB (two CTAs per SM), else two at
    // one CTA per SM (a 108 KB budget, 4 buffers at d=120, measured 7 % slower)
    int nbuf = 0;
    for (int n = 4; n >= 2 && !nbuf; --n)
        if (trace_tile_smem(n, kcap) <= 104 * 1024) nbuf = n;
    if (!nbuf && trace_tile_smem(2, kcap) + 4096 <= (size_t)max_smem_optin(P)) nbuf = 2;
    if (!nbuf) return GRAPE_OK;
    int4 *dblk = nullptr, *drun = nullptr;
    uint4 *dnb = nullptr;
    grape_status st;
    if ((st = upload(P, blk, &dblk)) != GRAPE_OK) return st;
    if ((st = upload(P, runs, &drun)) != GRAPE_OK) return st;
    if ((st = upload(P, nb, &dnb)) != GRAPE_OK) return st;
    t->tblk = dblk;
    t->trun = drun;
    t->tnb = dnb;
    t->kcap = kcap;
    t->nbuf = nbuf;
    t->tile = 1;
    return GRAPE_OK;
}

// largest segment (halving from the whole problem) whose storage fits the budget
long long seg_for_budget(const grape_problem *P, size_t budget) {
    long long seg = P->n_slices;
    while (seg > 1 && seg_bytes(P, seg) > budget) seg = (seg + 1) / 2;
    return seg;
}

// The adjoint sweep of a segment runs in chunks of slices; the trace kernel
// of each finished chunk runs on the problem's second stream while the next
// chunk propagates, on the SMs the propagation leaves idle.
int adjoint_chunks(const grape_problem *P, long long j0, long long j1, bool concurrent = false) {
    // concurrent sweeps: finer chunks shorten the traces left after both sweeps
    int n = concurrent ? 16 : 8;
    if (const char *env = std::getenv("GRAPE_ADJ_CHUNKS")) n = std::atoi(env);
    n = std::max(1, std::min(n, grape_problem::kMaxChunks));
    return (int)std::min<long long>(n, j1 - j0);
}

// Whether grape_gradient runs the forward and the adjoint sweep at the same
// time.  The cost Phi = sum_s Re Tr(sigma_s rho_s(T)) and the running
// penalty are linear in rho, so the adjoint's start value (sigma, plus the
// penalty's constant diagonal) and the exact discrete adjoint recursion
// (the transpose of the RK4 propagator, Eq. partialuk) never read the
// forward states: only the traces pair the two sweeps.  The forward sweep
// then runs in the adjoint's chunks, and the trace of chunk c waits for both
// sweeps to pass it.  Exact mode with the whole problem in one segment, on a
// cluster kernel (the grid kernel's per-problem stage buffers and flags admit
// one sweep at a time); GRAPE_CONCURRENT=0 turns it off.  Same kernels, same
// arithmetic: the same bits.
bool concurrent_sweeps(const grape_problem *P, int nseg) {
    if (P->mode != GRAPE_GRAD_EXACT || nseg != 1 || P->grid) return false;
    if (const char *env = std::getenv("GRAPE_CONCURRENT"))
        if (std::atoi(env) == 0) return false;
    if (const char *env = std::getenv("GRAPE_TRACE_OVERLAP"))
        if (std::atoi(env) == 0) return false;
    return true;
}

int gradient_launch_count(const grape_problem *P, int seg, int nseg, bool concurrent = false) {
    if (nseg <= 0) return -1;
    int n = 2;                                    // forward sweep, cost
    if (concurrent) n += adjoint_chunks(P, 0, P->n_slices, true) - 1;   // the forward in chunks
    if (P->penalty) n += 3;                       // adjoint start, final-state value, sum
    for (int gi = 0; gi < nseg; ++gi) {
        const long long j0 = (long long)gi * seg;
        const long long j1 = std::min<long long>(P->n_slices, j0 + seg);
        const int nch = adjoint_chunks(P, j0, j1, concurrent);
        n += (nseg > 1 ? 1 : 0) + nch;
        if (P->R > 0) n += nch * (P->trace.nsplit > 1 ? 2 : 1);
        if (P->penalty) n += 1;                   // boundary values of the segment
    }
    return n;
}

grape_status plan_gradient(grape_problem *P, size_t budget_override = 0) {
    if (P->nseg > 0) return GRAPE_OK;
    size_t free_b = 0, total_b = 0;
    GRAPE_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
    double frac = 0.6;
    if (const char *env = std::getenv("GRAPE_MEM_FRACTION")) {
        const double v = std::atof(env);
        if (v > 0.0 && v <= 0.95) frac = v;
    }
    const size_t budget = budget_override ? budget_override : (size_t)(frac * (double)free_b);
    long long seg;
    if (P->ckpt_stride > 0) {
        seg = std::min<long long>(P->ckpt_stride, P->n_slices);
    } else {
        seg = P->n_slices;
        while (seg > 1 && seg_bytes(P, seg) > budget) seg = (seg + 1) / 2;
    }
    if (seg_bytes(P, seg) > budget && P->ckpt_stride <= 0)
        return fail(GRAPE_ENOMEM, "gradient storage does not fit in device memory");
    const size_t per = stage_bytes(P, seg);
    P->d_Y = static_cast<double2 *>(P->alloc_grad(per));
    P->d_K = static_cast<double2 *>(P->alloc_grad(per));
    if (!P->d_Y || !P->d_K) return fail(GRAPE_ENOMEM, "cudaMalloc failed for gradient storage");
    const int nseg = (int)((P->n_slices + seg - 1) / seg);
    if (nseg > 1) {
        P->d_ckpt = static_cast<double2 *>(P->alloc_grad(ckpt_bytes(P, seg)));
        if (!P->d_ckpt) return fail(GRAPE_ENOMEM, "cudaMalloc failed for checkpoints");
    }
    P->seg = (int)seg;
    P->nseg = nseg;
    return GRAPE_OK;
}

enum { PH_FORWARD = 0, PH_COST = 1, PH_ADJOINT = 2, PH_TRACE = 3 };

// Runs one launch, bracketed by CUDA events on its stream when profiling.
template <typename F>
grape_status timed(grape_problem *P, int phase, cudaStream_t s, F &&launch) {
    cudaEvent_t a = nullptr, b = nullptr;
    if (P->profiling) {
        a = P->take_event();
        b = P->take_event();
        if (a) cudaEventRecord(a, s);
    }
    const cudaError_t e = launch();
    if (P->profiling && a && b) {
        cudaEventRecord(b, s);
        P->marks.push_back({phase, a, b});
    }
    if (e != cudaSuccess) return fail(GRAPE_ECUDA, std::string("kernel launch: ") + cudaGetErrorString(e));
    return GRAPE_OK;
}

grape_status launch_prop(grape_problem *P, const PropArgs &a, cudaStream_t s) {
    return timed(P, a.reverse ? PH_ADJOINT : PH_FORWARD, s,
                 [&] { return k_prop(P, a, s); });
}

grape_status stage_inputs(grape_problem *P, const double *u, const double **u_dev,
                          cudaStream_t s) {
    const size_t ub = (size_t)P->n_slices * P->R * sizeof(double);
    if (P->R == 0) { *u_dev = P->d_u; return GRAPE_OK; }
    if (!u) return fail(GRAPE_EINVAL, "u is NULL");
    bool on_dev = false;
    grape_status st = locate_ptr(u, P->device, "u", &on_dev);
    if (st != GRAPE_OK) return st;
    if (on_dev) {
        *u_dev = u;
    } else {
        GRAPE_CUDA_TRY(cudaMemcpyAsync(P->d_u, u, ub, cudaMemcpyHostToDevice, s));
        *u_dev = P->d_u;
    }
    return GRAPE_OK;
}

}  // namespace

// Running-cost penalty launches (App. B).  pen_rows: Re Tr(A rho_n) for
// `rows` consecutive boundary states stored `stride` entries apart (packed:
// upper triangles, as in the exact gradient's stage storage).
grape_status pen_rows(grape_problem *P, const void *x, long long stride, long long rows, long long first,
                      cudaStream_t s, int packed = 0) {
    GRAPE_CUDA_TRY(P->prec == GRAPE_PREC_FP64
                       ? grape_launch_penalty_rows_f64(x, stride, (int)rows, P->ns, P->d, P->d_pdiag,
                                                       P->d_pen + first, packed, s)
                       : grape_launch_penalty_rows_df(x, stride, (int)rows, P->ns, P->d, P->d_pdiag,
                                                      P->d_pen + first, packed, s));
    return GRAPE_OK;
}
grape_status pen_finish(grape_problem *P, double *F, cudaStream_t s) {
    const double scale = P->pen_beta * P->T / P->n_slices;
    GRAPE_CUDA_TRY(P->prec == GRAPE_PREC_FP64
                       ? grape_launch_penalty_finish_f64(P->d_pen, P->n_slices + 1, scale, F, s)
                       : grape_launch_penalty_finish_df(P->d_pen, P->n_slices + 1, scale, F, s));
    return GRAPE_OK;
}

// The trace kernels (Eq. dphidu) of slices [cA, cB), whose stage storage
// starts kofs entries into S.Y and S.K, on stream ts.
grape_status trace_chunk(grape_problem *P, const GradScratch &S, double *Gd, long long cA, long long cB,
                         size_t kofs, cudaStream_t ts) {
    grape_status st;
    const bool exact = (P->mode == GRAPE_GRAD_EXACT);
    const size_t mat = full_set(P);
    TraceArgs t = P->trace;
    t.n_rows = (int)(cB - cA);
    t.G = Gd + (size_t)cA * P->R;
    if (exact) {
        t.K = S.K + kofs;
        t.Y = S.Y + kofs;
        t.npairs = (long long)P->n_rk * 4 * P->ns;
        t.weight = 1.0;
    } else {
        t.K = S.K + kofs + mat;   // lambda_{j+1}, rho_{j+1} pair with row j
        t.Y = S.Y + kofs + mat;
        t.npairs = P->ns;
        t.weight = P->T / P->n_slices;
    }
    if (!S.part && !t.packed) t.nsplit = 1;
    t.part = S.part ? S.part + (size_t)cA * t.nsplit * P->R : nullptr;
    if ((st = timed(P, PH_TRACE, ts, [&] { return k_trace(P, t, ts); })) != GRAPE_OK) return st;
    if (t.nsplit > 1 &&
        (st = timed(P, PH_TRACE, ts, [&] {
             return P->prec == GRAPE_PREC_FP64 ? grape_launch_trace_finish_f64(t, ts)
                                               : grape_launch_trace_finish_df(t, ts);
         })) != GRAPE_OK)
        return st;
    return GRAPE_OK;
}

// The gradient with the forward and the adjoint sweep at the same time (see
// concurrent_sweeps): the forward in the adjoint's chunks on s (then the
// cost and the running penalty's rows), the adjoint on S.s3 (start value,
// chunks last first), the trace of chunk c on S.s2 once both sweeps have
// passed it; s then waits for both.
grape_status run_gradient_concurrent(grape_problem *P, const double *ud, double *Fd, double *Gd,
                                     cudaStream_t s, const GradScratch &S) {
    grape_status st;
    const size_t mat = full_set(P);
    const size_t pst = packed_set(P);
    const long long j0 = 0, j1 = P->n_slices;
    const int nch = adjoint_chunks(P, j0, j1, true);
    const size_t per_slice = (size_t)P->n_rk * 4 * pst;   // stored stage entries per slice
    cudaStream_t sa = S.s3, ts = S.s2;
    GRAPE_CUDA_TRY(cudaEventRecord(S.fork3, s));
    GRAPE_CUDA_TRY(cudaStreamWaitEvent(sa, S.fork3, 0));
    // adjoint start value: sigma (and the penalty's last term)
    GRAPE_CUDA_TRY(cudaMemcpyAsync(S.mu, P->d_sigma, mat * sizeof(double2), cudaMemcpyDeviceToDevice, sa));
    if (P->penalty)
        GRAPE_CUDA_TRY(P->prec == GRAPE_PREC_FP64 ? grape_launch_add_diag_f64(S.mu, P->d_src, P->d, P->ns, sa)
                                                  : grape_launch_add_diag_df(S.mu, P->d_src, P->d, P->ns, sa));
    // forward sweep in chunks, each storing its slices' stage inputs
    for (int ci = 0; ci < nch; ++ci) {
        const long long cA = j0 + (j1 - j0) * ci / nch;
        const long long cB = j0 + (j1 - j0) * (ci + 1) / nch;
        PropArgs f = base_args(P, 0, ud);
        f.sub_begin = cA * P->n_rk;
        f.sub_end = cB * P->n_rk;
        f.x_in = ci == 0 ? P->d_rho0 : S.x;
        f.x_out = S.x;
        f.stage_store = S.Y + (size_t)(cA - j0) * per_slice;
        if ((st = launch_prop(P, f, s)) != GRAPE_OK) return st;
        GRAPE_CUDA_TRY(cudaEventRecord(S.evF[ci], s));
    }
    if ((st = timed(P, PH_COST, s, [&] { return k_cost(P, S.x, Fd, s); })) != GRAPE_OK) return st;
    if (P->penalty) {
        if ((st = pen_rows(P, S.x, 0, 1, P->n_slices, s)) != GRAPE_OK) return st;
        if ((st = pen_rows(P, S.Y, (long long)per_slice, j1 - j0, j0, s, 1)) != GRAPE_OK) return st;
    }
    // adjoint chunks (last slices first)
    for (int ci = nch - 1; ci >= 0; --ci) {
        const long long cA = j0 + (j1 - j0) * ci / nch;
        const long long cB = j0 + (j1 - j0) * (ci + 1) / nch;
        PropArgs b = base_args(P, 1, ud);
        b.sub_begin = cA * P->n_rk;
        b.sub_end = cB * P->n_rk;
        b.reverse = 1;
        b.x_in = S.mu;
        b.x_out = S.mu;
        b.stage_store = S.K + (size_t)(cA - j0) * per_slice;
        if ((st = launch_prop(P, b, sa)) != GRAPE_OK) return st;
        GRAPE_CUDA_TRY(cudaEventRecord(S.ev[ci], sa));
    }
    // the traces in the order the chunks become ready: the forward passes
    // chunk c after c + 1 chunks, the adjoint after nch - c, so the middle
    // chunks are ready first and the two ends last (one in-order stream)
    int order[grape_problem::kMaxChunks];
    for (int c = 0; c < nch; ++c) order[c] = c;
    std::sort(order, order + nch, [nch](int a, int b) {
        const int ra = std::max(a + 1, nch - a), rb = std::max(b + 1, nch - b);
        return ra != rb ? ra < rb : a < b;
    });
    for (int k = 0; k < nch && P->R > 0; ++k) {
        const int ci = order[k];
        const long long cA = j0 + (j1 - j0) * ci / nch;
        const long long cB = j0 + (j1 - j0) * (ci + 1) / nch;
        GRAPE_CUDA_TRY(cudaStreamWaitEvent(ts, S.ev[ci], 0));
        GRAPE_CUDA_TRY(cudaStreamWaitEvent(ts, S.evF[ci], 0));
        if ((st = trace_chunk(P, S, Gd, cA, cB, (size_t)(cA - j0) * per_slice, ts)) != GRAPE_OK) return st;
    }
    GRAPE_CUDA_TRY(cudaEventRecord(S.ev[grape_problem::kMaxChunks + 1], sa));
    GRAPE_CUDA_TRY(cudaStreamWaitEvent(s, S.ev[grape_problem::kMaxChunks + 1], 0));
    if (P->R > 0) {
        GRAPE_CUDA_TRY(cudaEventRecord(S.ev[grape_problem::kMaxChunks], ts));
        GRAPE_CUDA_TRY(cudaStreamWaitEvent(s, S.ev[grape_problem::kMaxChunks], 0));
    }
    if (P->penalty) return pen_finish(P, Fd, s);     // Phi = Phi_0 - beta dt sum_n Tr(A rho_n)
    return GRAPE_OK;
}

// One gradient evaluation on stream s with device pointers only: forward
// sweep (stage storage or checkpoints), cost, then per segment (last first)
// the recomputed forward stage inputs, the adjoint sweep in chunks and the
// trace kernels of the finished chunks.
grape_status run_gradient(grape_problem *P, const double *ud, double *Fd, double *Gd,
                          cudaStream_t s, const GradScratch &S) {
    if (S.s3 && S.s2 && S.evF && concurrent_sweeps(P, S.nseg))
        return run_gradient_concurrent(P, ud, Fd, Gd, s, S);
    grape_status st;
    const bool exact = (P->mode == GRAPE_GRAD_EXACT);
    const long long nsub = (long long)P->n_slices * P->n_rk;
    const size_t mat = full_set(P);                  // a state set as full matrices
    const size_t pst = exact ? packed_set(P) : mat;  // a stored stage set (packed in exact mode)

    // forward sweep: stage storage directly (one segment) or checkpoints
    PropArgs f = base_args(P, 0, ud);
    f.sub_begin = 0;
    f.sub_end = nsub;
    f.x_in = P->d_rho0;
    f.x_out = S.x;
    if (S.nseg == 1) {
        if (exact) f.stage_store = S.Y;
        else { f.bound_store = S.Y; f.bound_step = P->n_rk; }
    } else {
        f.bound_store = S.ckpt;
        f.bound_step = (long long)S.seg * P->n_rk;
    }
    if ((st = launch_prop(P, f, s)) != GRAPE_OK) return st;
    if ((st = timed(P, PH_COST, s, [&] {
             return k_cost(P, S.x, Fd, s);
         })) != GRAPE_OK)
        return st;
    GRAPE_CUDA_TRY(cudaMemcpyAsync(S.mu, P->d_sigma, mat * sizeof(double2),
                                   cudaMemcpyDeviceToDevice, s));
    // boundary state n of a segment in the stage storage: the input of the
    // slice's first stage (exact mode) or the stored boundary (first order)
    const long long bstride = (long long)(exact ? (size_t)P->n_rk * 4 * pst : mat);
    if (P->penalty) {
        GRAPE_CUDA_TRY(P->prec == GRAPE_PREC_FP64
                           ? grape_launch_add_diag_f64(S.mu, P->d_src, P->d, P->ns, s)
                           : grape_launch_add_diag_df(S.mu, P->d_src, P->d, P->ns, s));
        if ((st = pen_rows(P, S.x, 0, 1, P->n_slices, s)) != GRAPE_OK) return st;
    }
    for (int gi = S.nseg - 1; gi >= 0; --gi) {
        const long long j0 = (long long)gi * S.seg;
        const long long j1 = std::min<long long>(P->n_slices, j0 + S.seg);
        if (S.nseg > 1) {   // recompute the segment's forward stage inputs from its checkpoint
            PropArgs r = base_args(P, 0, ud);
            r.sub_begin = j0 * P->n_rk;
            r.sub_end = j1 * P->n_rk;
            r.x_in = S.ckpt + (size_t)gi * mat;
            r.x_out = S.x;
            if (exact) r.stage_store = S.Y;
            else { r.bound_store = S.Y; r.bound_step = P->n_rk; }
            if ((st = launch_prop(P, r, s)) != GRAPE_OK) return st;
        }
        if (P->penalty && (st = pen_rows(P, S.Y, bstride, j1 - j0, j0, s, exact ? 1 : 0)) != GRAPE_OK)
            return st;
        // adjoint sweep in chunks (last slices first); the trace of each
        // finished chunk runs on s2, overlapping the next chunk
        const int nch = adjoint_chunks(P, j0, j1);
        for (int ci = nch - 1; ci >= 0; --ci) {
            const long long cA = j0 + (j1 - j0) * ci / nch;
            const long long cB = j0 + (j1 - j0) * (ci + 1) / nch;
            const size_t kofs = exact ? (size_t)(cA - j0) * P->n_rk * 4 * pst : (size_t)(cA - j0) * mat;
            PropArgs b = base_args(P, 1, ud);
            b.sub_begin = cA * P->n_rk;
            b.sub_end = cB * P->n_rk;
            b.reverse = 1;
            b.x_in = S.mu;
            b.x_out = S.mu;
            if (exact) b.stage_store = S.K + kofs;
            else { b.bound_store = S.K + kofs; b.bound_step = P->n_rk; }
            if ((st = launch_prop(P, b, s)) != GRAPE_OK) return st;
            if (P->R == 0) continue;
            cudaStream_t ts = S.s2 ? S.s2 : s;
            if (S.s2) {
                GRAPE_CUDA_TRY(cudaEventRecord(S.ev[ci], s));
                GRAPE_CUDA_TRY(cudaStreamWaitEvent(S.s2, S.ev[ci], 0));
            }
            if ((st = trace_chunk(P, S, Gd, cA, cB, kofs, ts)) != GRAPE_OK) return st;
        }
        if (P->R > 0 && S.s2) {   // the segment's stage storage is reused next: join s2 into s
            GRAPE_CUDA_TRY(cudaEventRecord(S.ev[grape_problem::kMaxChunks], S.s2));
            GRAPE_CUDA_TRY(cudaStreamWaitEvent(s, S.ev[grape_problem::kMaxChunks], 0));
        }
    }
    if (P->penalty) return pen_finish(P, Fd, s);     // Phi = Phi_0 - beta dt sum_n Tr(A rho_n)
    return GRAPE_OK;
}

extern "C" {

const char *grape_last_error(void) { return g_last_error.c_str(); }

const char *grape_version(void) { return "grape-gb300 0.3 (sm_103a, df64/fp64)"; }

grape_status grape_fma_peak(int32_t precision, double *tflops, double *ms) {
    if (!tflops || !ms) return fail(GRAPE_EINVAL, "NULL tflops or ms");
    if (precision != GRAPE_PREC_DF64 && precision != GRAPE_PREC_FP64)
        return fail(GRAPE_EINVAL, "unknown precision");
    GRAPE_CUDA_TRY(grape_probe_fma(precision, tflops, ms));
    return GRAPE_OK;
}

grape_status grape_problem_create(const grape_problem_desc *desc, grape_problem_t *out) {
    if (!desc || !out) return fail(GRAPE_EINVAL, "NULL descriptor or output");
    *out = nullptr;
    const int d = desc->d;
    if (d < 1 || d > 4096) return fail(GRAPE_EINVAL, "d must be in [1, 4096]");
    if (desc->n_controls < 0 || desc->n_controls > GRAPE_MAXR)
        return fail(GRAPE_EINVAL, "n_controls must be in [0, 8]");
    if (desc->n_jumps < 0 || desc->n_states < 1 || desc->n_slices < 1 || desc->n_rk < 1)
        return fail(GRAPE_EINVAL, "n_jumps >= 0, n_states >= 1, n_slices >= 1, n_rk >= 1 required");
    if (!(desc->T > 0.0) || !std::isfinite(desc->T)) return fail(GRAPE_EINVAL, "T must be positive");
    if (desc->grad_mode != GRAPE_GRAD_EXACT && desc->grad_mode != GRAPE_GRAD_FIRST_ORDER)
        return fail(GRAPE_EINVAL, "unknown grad_mode");
    if (desc->ckpt_stride < 0) return fail(GRAPE_EINVAL, "ckpt_stride must be >= 0");
    if (desc->precision != GRAPE_PREC_DF64 && desc->precision != GRAPE_PREC_FP64)
        return fail(GRAPE_EINVAL, "unknown precision");
    if (!desc->rho0 || !desc->sigma) return fail(GRAPE_EINVAL, "rho0 and sigma are required");
    if (desc->n_controls > 0 && !desc->Hc) return fail(GRAPE_EINVAL, "Hc is NULL");
    if (desc->n_jumps > 0 && (!desc->jumps || !desc->rates)) return fail(GRAPE_EINVAL, "jumps/rates NULL");

    grape_status st;
    Bands H0;
    if ((st = read_bands(desc->H0, d, "H0", &H0)) != GRAPE_OK) return st;
    if (!hermitian(H0, d)) return fail(GRAPE_EINVAL, "H0 is not Hermitian");
    std::vector<Bands> Hc(desc->n_controls);
    for (int k = 0; k < desc->n_controls; ++k) {
        if ((st = read_bands(desc->Hc[k], d, "Hc", &Hc[k])) != GRAPE_OK) return st;
        if (!hermitian(Hc[k], d)) return fail(GRAPE_EINVAL, "a control Hamiltonian is not Hermitian");
        prune(Hc[k]);
    }
    std::vector<Bands> C(desc->n_jumps);
    for (int m = 0; m < desc->n_jumps; ++m) {
        const double g = desc->rates[m];
        if (!(g >= 0.0) || !std::isfinite(g)) return fail(GRAPE_EINVAL, "rates must be finite and >= 0");
        if ((st = read_bands(desc->jumps[m], d, "jump", &C[m])) != GRAPE_OK) return st;
        prune(C[m]);
    }

    // controls on dissipation rates
    std::vector<int> jc(desc->n_jumps, -1);
    if (desc->jump_control)
        for (int m = 0; m < desc->n_jumps; ++m) {
            const int k = desc->jump_control[m];
            if (k < -1 || k >= desc->n_controls) return fail(GRAPE_EINVAL, "jump_control out of range");
            if (k >= 0 && !Hc[k].empty())
                return fail(GRAPE_EINVAL, "a control on a dissipation rate must have an empty Hamiltonian");
            jc[m] = k;
        }
    // Forward: A = H_eff = H0 - i/2 sum gamma c^+ c (+ sum u_k A_k), terms from sqrt(gamma) c.
    // A rate control k contributes A_k = -i/2 gamma c^+ c and scales its terms by u_k.
    Bands A0 = H0;
    std::vector<Bands> Ak = Hc;                 // propagation's control parts
    std::vector<Bands> Tk = Hc;                 // trace's control bands (see below)
    std::vector<Bands> Jf, Ja;
    std::vector<int> jcf;
    for (int m = 0; m < desc->n_jumps; ++m) {
        const double g = desc->rates[m];
        if (g == 0.0 || C[m].empty()) continue;
        const Bands cdc = product(adjoint(C[m], d), C[m], d);
        if (jc[m] < 0) {
            add_into(A0, cdc, cplx(0.0, -0.5 * g), d);
        } else {
            add_into(Ak[jc[m]], cdc, cplx(0.0, -0.5 * g), d);
            // -1/2 gamma {c^+c, y} enters Re Tr(kb dL/du y) as the commutator
            // term of the trace kernel does with the band values +i/2 gamma c^+c
            add_into(Tk[jc[m]], cdc, cplx(0.0, 0.5 * g), d);
        }
        Jf.push_back(scaled(C[m], std::sqrt(g), d));
        Ja.push_back(scaled(adjoint(C[m], d), std::sqrt(g), d));
        jcf.push_back(jc[m]);
    }
    prune(A0);
    for (auto &b : Ak) prune(b);
    for (auto &b : Tk) prune(b);
    // Dual: A' = -H_eff^+, A'_k = -A_k^+, terms from sqrt(gamma) c^+.
    Bands A0d = scaled(adjoint(A0, d), -1.0, d);
    std::vector<Bands> Hcd(Ak.size());
    for (size_t k = 0; k < Ak.size(); ++k) Hcd[k] = scaled(adjoint(Ak[k], d), -1.0, d);
    for (auto &c : Jf) prune(c);
    for (auto &c : Ja) prune(c);
    const HostDir hf = make_dir(A0, Ak, Jf, jcf, d);
    const HostDir ha = make_dir(A0d, Hcd, Ja, jcf, d);

    // initial states (Hermitian) and the Hermitian part of sigma
    const size_t d2 = (size_t)d * d;
    std::vector<cplx> rho0(d2 * desc->n_states), sig(d2 * desc->n_states);
    for (int s = 0; s < desc->n_states; ++s) {
        const double *r = desc->rho0 + 2 * d2 * s;
        double mx = 0.0, asym = 0.0;
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) {
                const cplx a(r[2 * (i * d + j)], r[2 * (i * d + j) + 1]);
                const cplx b(r[2 * (j * d + i)], r[2 * (j * d + i) + 1]);
                if (!std::isfinite(a.real()) || !std::isfinite(a.imag()))
                    return fail(GRAPE_EINVAL, "rho0 has non-finite entries");
                mx = std::max(mx, std::abs(a));
                asym = std::max(asym, std::abs(a - std::conj(b)));
                rho0[s * d2 + i * d + j] = a;
            }
        if (asym > 1e-12 * std::max(mx, 1e-300)) return fail(GRAPE_EINVAL, "rho0 is not Hermitian");
        const double *g = desc->sigma + (desc->sigma_broadcast ? 0 : 2 * d2 * s);
        for (int i = 0; i < d; ++i)
            for (int j = 0; j < d; ++j) {
                const cplx a(g[2 * (i * d + j)], g[2 * (i * d + j) + 1]);
                const cplx b(g[2 * (j * d + i)], g[2 * (j * d + i) + 1]);
                if (!std::isfinite(a.real()) || !std::isfinite(a.imag()))
                    return fail(GRAPE_EINVAL, "sigma has non-finite entries");
                const cplx hpart = 0.5 * (a + std::conj(b));
                sig[s * d2 + i * d + j] = hpart;
            }
    }

    // control bands for the trace kernel
    TraceArgs tr;
    std::memset(&tr, 0, sizeof(tr));
    std::vector<double2> cbv, stv_l, stv_r;
    {
        std::map<int, int> doidx;
        for (int k = 0; k < desc->n_controls; ++k)
            for (const auto &kv : Tk[k]) {
                if (tr.ncb >= GRAPE_MAXCB) return fail(GRAPE_EINVAL, "too many control bands (max 8)");
                auto it = doidx.find(kv.first);
                if (it == doidx.end()) {
                    if ((int)doidx.size() >= GRAPE_MAXDO) return fail(GRAPE_EINVAL, "too many control band offsets");
                    const int id = (int)doidx.size();
                    doidx[kv.first] = id;
                    tr.do_off[id] = kv.first;
                    it = doidx.find(kv.first);
                }
                tr.cb_k[tr.ncb] = k;
                tr.cb_do[tr.ncb] = it->second;
                for (int i = 0; i < d; ++i) cbv.push_back(make_double2(kv.second[i].real(), kv.second[i].imag()));
                tr.ncb++;
            }
        tr.ndo = (int)doidx.size();
        tr.d = d;
        tr.R = desc->n_controls;
        // sandwich terms gamma c y c^+ of the rate-controlled dissipators: the
        // forward jump terms (sqrt(gamma) c on both sides) of those dissipators
        for (size_t q = 0; q < hf.oL.size(); ++q) {
            if (hf.jctl[q] < 0) continue;
            if (tr.nst >= GRAPE_MAXST)
                return fail(GRAPE_EINVAL, "too many band pairs in rate-controlled dissipators (max 4)");
            tr.st_k[tr.nst] = hf.jctl[q];
            tr.st_oL[tr.nst] = hf.oL[q];
            tr.st_oR[tr.nst] = hf.oR[q];
            for (int i = 0; i < d; ++i) {
                stv_l.push_back(make_double2(hf.vL[q * d + i].real(), hf.vL[q * d + i].imag()));
                stv_r.push_back(make_double2(hf.vR[q * d + i].real(), hf.vR[q * d + i].imag()));
            }
            tr.nst++;
        }
    }

    grape_problem *P = new grape_problem();
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        delete P;
        return fail(GRAPE_ECUDA, "no CUDA device");
    }
    P->device = dev;
    static_scratch_setup(dev);   // grape_gradient_static's array, committed once per device
    P->d = d;
    P->d2 = d2;
    P->R = desc->n_controls;
    P->J = desc->n_jumps;
    P->ns = desc->n_states;
    P->n_slices = desc->n_slices;
    P->n_rk = desc->n_rk;
    P->T = desc->T;
    P->mode = desc->grad_mode;
    P->ckpt_stride = desc->ckpt_stride;
    P->prec = desc->precision;
    auto bail = [&](grape_status s) { delete P; return s; };
    {
        // real jump tables select the kernels with one real coefficient per
        // term; rate-controlled terms always take the complex-table kernels,
        // which alone carry the per-slice scaling
        bool real_jumps = true;
        for (const HostDir *h : {&hf, &ha})
            for (const auto *v : {&h->vL, &h->vR})
                for (const cplx &c : *v) real_jumps = real_jumps && c.imag() == 0.0;
        for (int c : jcf) real_jumps = real_jumps && c < 0;
        P->variant = real_jumps ? 1 : 0;
    }
    // error word of the bounded waits (grid barrier arrivals, generation, flag)
    P->d_gbar = static_cast<unsigned *>(P->alloc(4 * sizeof(unsigned)));
    if (!P->d_gbar) return bail(fail(GRAPE_ENOMEM, "cudaMalloc failed for the error word"));
    if (cudaMemset(P->d_gbar, 0, 4 * sizeof(unsigned)) != cudaSuccess ||
        cudaStreamSynchronize(cudaStreamLegacy) != cudaSuccess) {   // before non-blocking streams use it
        cudaGetLastError();
        return bail(fail(GRAPE_ECUDA, "cudaMemset of the error word failed"));
    }
    if ((st = upload_dir(P, hf, &P->tab[0])) != GRAPE_OK) return bail(st);
    if ((st = upload_dir(P, ha, &P->tab[1])) != GRAPE_OK) return bail(st);
    int omax = 0;
    for (int dir = 0; dir < 2; ++dir) {
        const HostDir &h = dir ? ha : hf;
        for (int o : h.off) omax = std::max(omax, std::abs(o));
        for (size_t q = 0; q < h.oL.size(); ++q)
            omax = std::max(omax, std::max(std::abs(h.oL[q]), std::abs(h.oR[q])));
    }
    int hb = omax;   // lower entries the stencil reads: within max(omax, oL - oR) of the diagonal
    for (int dir = 0; dir < 2; ++dir) {
        const HostDir &h = dir ? ha : hf;
        for (size_t q = 0; q < h.oL.size(); ++q) hb = std::max(hb, h.oL[q] - h.oR[q]);
    }
    // kernel choice: Hermitian cluster kernel, else full-matrix cluster kernel,
    // else the grid kernel (GRAPE_KERNEL=grid|cluster|full forces one)
    std::string kern = "auto";
    if (const char *env = std::getenv("GRAPE_KERNEL")) kern = env;
    bool herm = kern == "auto" || kern == "cluster";
    if (const char *env = std::getenv("GRAPE_HERMITIAN")) herm = herm && std::atoi(env) != 0;
    bool placed = false;
    P->omax = omax;
    P->hb_h = hb;
    if (kern != "grid" && herm) {
        st = choose_geometry_h(P);
        if (st != GRAPE_OK && st != GRAPE_EINVAL) return bail(st);
        placed = (st == GRAPE_OK);
    }
    if (kern != "grid" && !placed) {
        st = choose_geometry(P);
        if (st != GRAPE_OK && st != GRAPE_EINVAL) return bail(st);
        placed = (st == GRAPE_OK);
    }
    if (!placed && (st = choose_geometry_grid(P)) != GRAPE_OK) return bail(st);
    {
        std::vector<double2> r(rho0.size()), g2(sig.size());
        for (size_t i = 0; i < r.size(); ++i) r[i] = encode(P, rho0[i]);
        for (size_t i = 0; i < g2.size(); ++i) g2[i] = encode(P, sig[i]);
        if ((st = upload(P, r, &P->d_rho0)) != GRAPE_OK) return bail(st);
        if ((st = upload(P, g2, &P->d_sigma)) != GRAPE_OK) return bail(st);
    }
    // the kernels read the tables in their storage format (no conversion
    // from FP64 in the double-float build)
    auto to_store = [&](const std::vector<double2> &v) {
        std::vector<double2> o(v.size());
        for (size_t i = 0; i < v.size(); ++i) o[i] = encode(P, cplx(v[i].x, v[i].y));
        return o;
    };
    double2 *cbs = nullptr;
    if ((st = upload(P, to_store(cbv), &cbs)) != GRAPE_OK) return bail(st);
    tr.cb_s = cbs;
    if (tr.nst > 0) {
        double2 *as = nullptr, *bs = nullptr;
        if ((st = upload(P, to_store(stv_l), &as)) != GRAPE_OK) return bail(st);
        if ((st = upload(P, to_store(stv_r), &bs)) != GRAPE_OK) return bail(st);
        tr.st_vLs = as;
        tr.st_vRs = bs;
    }
    P->trace = tr;
    trace_layout(P, &P->trace);
    if ((st = trace_tiles(P, &P->trace)) != GRAPE_OK) return bail(st);

    P->d_x = static_cast<double2 *>(P->alloc(d2 * P->ns * sizeof(double2)));
    P->d_mu = static_cast<double2 *>(P->alloc(d2 * P->ns * sizeof(double2)));
    P->d_out = static_cast<double2 *>(P->alloc(d2 * P->ns * sizeof(double2)));
    P->d_part = static_cast<double *>(
        P->alloc((size_t)P->n_slices * P->trace.nsplit * std::max(P->R, 1) * sizeof(double)));
    P->d_u = static_cast<double *>(P->alloc((size_t)P->n_slices * std::max(P->R, 1) * sizeof(double)));
    P->d_F = static_cast<double *>(P->alloc(sizeof(double)));
    P->d_G = static_cast<double *>(P->alloc((size_t)P->n_slices * std::max(P->R, 1) * sizeof(double)));
    if (!P->d_x || !P->d_mu || !P->d_out || !P->d_part || !P->d_u || !P->d_F || !P->d_G) return bail(fail(GRAPE_ENOMEM, "cudaMalloc failed"));
    {
        int prio_low = 0, prio_high = 0;
        cudaDeviceGetStreamPriorityRange(&prio_low, &prio_high);
        if (cudaStreamCreateWithPriority(&P->s1, cudaStreamNonBlocking, prio_high) != cudaSuccess ||
            cudaStreamCreateWithPriority(&P->s2, cudaStreamNonBlocking, prio_low) != cudaSuccess ||
            cudaStreamCreateWithPriority(&P->s3, cudaStreamNonBlocking, prio_high) != cudaSuccess ||
            cudaEventCreateWithFlags(&P->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&P->ev_fork3, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&P->ev_join, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return bail(fail(GRAPE_ECUDA, "cudaStreamCreate failed"));
        }
    }
    for (auto &e : P->ev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return bail(fail(GRAPE_ECUDA, "cudaEventCreate failed"));
        }
    for (auto &e : P->evF)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return bail(fail(GRAPE_ECUDA, "cudaEventCreate failed"));
        }
    *out = P;
    return GRAPE_OK;
}

grape_status grape_problem_destroy(grape_problem_t P) {
    if (!P) return GRAPE_OK;
    DeviceGuard g(P->device);
    delete P;
    return GRAPE_OK;
}

grape_status grape_problem_memory(grape_problem_t P, size_t *bytes) {
    if (!P || !bytes) return fail(GRAPE_EINVAL, "NULL argument");
    *bytes = P->bytes;
    return GRAPE_OK;
}

grape_status grape_problem_geometry(grape_problem_t P, int32_t *cluster, int32_t *threads,
                                    int32_t *ept) {
    if (!P) return fail(GRAPE_EINVAL, "NULL problem");
    if (cluster) *cluster = P->ncl;
    if (threads) *threads = P->threads;
    if (ept) *ept = (P->chunk + P->threads - 1) / P->threads;
    return GRAPE_OK;
}

grape_status grape_problem_set_penalty(grape_problem_t P, const double *diag, double beta) {
    if (!P) return fail(GRAPE_EINVAL, "NULL problem");
    if (!std::isfinite(beta)) return fail(GRAPE_EINVAL, "penalty weight must be finite");
    if (!diag || beta == 0.0) {
        P->penalty = false;
        P->pen_beta = 0.0;
        return GRAPE_OK;
    }
    for (int i = 0; i < P->d; ++i)
        if (!std::isfinite(diag[i])) return fail(GRAPE_EINVAL, "penalty operator entries must be finite");
    DeviceGuard g(P->device);
    const double dt = P->T / P->n_slices;
    std::vector<double> a(diag, diag + P->d), src(P->d);
    for (int i = 0; i < P->d; ++i) src[i] = -beta * dt * a[i];
    if (!P->d_pdiag) {
        P->d_pdiag = static_cast<double *>(P->alloc(P->d * sizeof(double)));
        P->d_src = static_cast<double *>(P->alloc(P->d * sizeof(double)));
        P->d_pen = static_cast<double *>(P->alloc((size_t)(P->n_slices + 1) * sizeof(double)));
        if (!P->d_pdiag || !P->d_src || !P->d_pen) return fail(GRAPE_ENOMEM, "cudaMalloc failed for the penalty");
    }
    // callers' kernels may still read the old values: order after the device
    GRAPE_CUDA_TRY(cudaDeviceSynchronize());
    GRAPE_CUDA_TRY(cudaMemcpy(P->d_pdiag, a.data(), P->d * sizeof(double), cudaMemcpyHostToDevice));
    GRAPE_CUDA_TRY(cudaMemcpy(P->d_src, src.data(), P->d * sizeof(double), cudaMemcpyHostToDevice));
    GRAPE_CUDA_TRY(cudaStreamSynchronize(cudaStreamLegacy));
    P->pen_beta = beta;
    P->penalty = true;
    return GRAPE_OK;
}

grape_status grape_problem_set_tile(grape_problem_t P, int32_t cluster, int32_t threads) {
    if (!P) return fail(GRAPE_EINVAL, "NULL problem");
    if (!(cluster == 1 || cluster == 2 || cluster == 4 || cluster == 8 || cluster == 16))
        return fail(GRAPE_EINVAL, "cluster width must be 1, 2, 4, 8 or 16");
    if (threads < 64 || threads > GRAPE_PROP_THREADS || threads % 32 != 0)
        return fail(GRAPE_EINVAL, "threads per CTA must be a multiple of 32 in [64, 512]");
    if (P->grid) return fail(GRAPE_EINVAL, "the grid kernel has no tile to set");
    DeviceGuard g(P->device);
    return (P->variant & 2) ? plan_h(P, cluster, threads) : plan_full(P, cluster, threads);
}

grape_status grape_problem_status(grape_problem_t P) {
    if (!P) return fail(GRAPE_EINVAL, "NULL problem");
    DeviceGuard g(P->device);
    unsigned flag[3] = {0, 0, 0};
    GRAPE_CUDA_TRY(cudaDeviceSynchronize());
    GRAPE_CUDA_TRY(cudaMemcpy(flag, P->d_gbar, sizeof(flag), cudaMemcpyDeviceToHost));
    if (flag[2] != 0u) {
        GRAPE_CUDA_TRY(cudaMemset(P->d_gbar, 0, 4 * sizeof(unsigned)));
        GRAPE_CUDA_TRY(cudaStreamSynchronize(cudaStreamLegacy));
        return fail(GRAPE_ETIMEOUT, flag[2] == 3u   ? "a copy wait of the staged trace kernel gave up waiting"
                                    : flag[2] == 2u ? "a window wait of the cluster propagation kernel gave up waiting"
                                                    : "a grid barrier of the propagation kernel gave up waiting");
    }
    return GRAPE_OK;
}

grape_status grape_problem_kernel(grape_problem_t P, int32_t *kind) {
    if (!P || !kind) return fail(GRAPE_EINVAL, "NULL argument");
    *kind = P->grid ? 2 : ((P->variant & 2) ? 0 : 1);
    return GRAPE_OK;
}

grape_status grape_set_profiling(grape_problem_t P, int32_t on) {
    if (!P) return fail(GRAPE_EINVAL, "NULL problem");
    P->profiling = (on != 0);
    return GRAPE_OK;
}

grape_status grape_phase_times(grape_problem_t P, double ms[4], int32_t launches[4]) {
    if (!P || !ms || !launches) return fail(GRAPE_EINVAL, "NULL argument");
    DeviceGuard g(P->device);
    for (int i = 0; i < 4; ++i) { ms[i] = 0.0; launches[i] = 0; }
    grape_status st = GRAPE_OK;
    for (auto &m : P->marks) {
        float t = 0.0f;
        cudaError_t e = cudaEventSynchronize(m.b);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&t, m.a, m.b);
        if (e != cudaSuccess && st == GRAPE_OK)
            st = fail(GRAPE_ECUDA, std::string("event timing: ") + cudaGetErrorString(e));
        ms[m.phase] += t;
        launches[m.phase] += 1;
        P->event_pool.push_back(m.a);
        P->event_pool.push_back(m.b);
    }
    P->marks.clear();
    return st;
}

int32_t grape_gradient_launches(grape_problem_t P) {
    if (!P) return -1;
    return gradient_launch_count(P, P->seg, P->nseg, concurrent_sweeps(P, P->nseg));
}

grape_status grape_forward(grape_problem_t P, const double *u, double *F, double *rhoT,
                           void *stream) {
    if (!P || !F) return fail(GRAPE_EINVAL, "NULL problem or F");
    DeviceGuard g(P->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const double *ud;
    grape_status st;
    bool f_dev = false, r_dev = false;
    if ((st = locate_ptr(F, P->device, "F", &f_dev)) != GRAPE_OK) return st;
    if ((st = locate_ptr(rhoT, P->device, "rhoT", &r_dev)) != GRAPE_OK) return st;
    if ((st = stage_inputs(P, u, &ud, s)) != GRAPE_OK) return st;
    PropArgs a = base_args(P, 0, ud);
    a.sub_begin = 0;
    a.sub_end = (long long)P->n_slices * P->n_rk;
    a.x_in = P->d_rho0;
    a.x_out = P->d_x;
    const size_t mat = P->d2 * P->ns;
    if (!P->penalty) {
        if ((st = launch_prop(P, a, s)) != GRAPE_OK) return st;
    } else {
        // the running cost needs every boundary state: chunks of kPenChunk
        // slices keep their boundaries in a small buffer
        if (!P->d_fwd_bounds) {
            P->d_fwd_bounds = static_cast<double2 *>(
                P->alloc((size_t)(grape_problem::kPenChunk + 1) * mat * sizeof(double2)));
            if (!P->d_fwd_bounds) return fail(GRAPE_ENOMEM, "cudaMalloc failed for boundary states");
        }
        for (long long j0 = 0; j0 < P->n_slices; j0 += grape_problem::kPenChunk) {
            const long long j1 = std::min<long long>(P->n_slices, j0 + grape_problem::kPenChunk);
            a.sub_begin = j0 * P->n_rk;
            a.sub_end = j1 * P->n_rk;
            a.x_in = j0 == 0 ? P->d_rho0 : P->d_x;
            a.bound_store = P->d_fwd_bounds;
            a.bound_step = P->n_rk;
            if ((st = launch_prop(P, a, s)) != GRAPE_OK) return st;
            if ((st = pen_rows(P, P->d_fwd_bounds, (long long)mat, j1 - j0, j0, s)) != GRAPE_OK) return st;
        }
        if ((st = pen_rows(P, P->d_x, 0, 1, P->n_slices, s)) != GRAPE_OK) return st;
    }
    if ((st = timed(P, PH_COST, s, [&] {
             return k_cost(P, P->d_x, f_dev ? F : P->d_F, s);
         })) != GRAPE_OK)
        return st;
    if (P->penalty && (st = pen_finish(P, f_dev ? F : P->d_F, s)) != GRAPE_OK) return st;
    bool sync = false;
    if (rhoT) {
        const size_t n = P->d2 * P->ns;
        GRAPE_CUDA_TRY(k_to_double(P, P->d_x, r_dev ? reinterpret_cast<double2 *>(rhoT) : P->d_out, n, s));
        if (!r_dev) {
            GRAPE_CUDA_TRY(cudaMemcpyAsync(rhoT, P->d_out, n * sizeof(double2), cudaMemcpyDeviceToHost, s));
            sync = true;
        }
    }
    if (!f_dev) {
        GRAPE_CUDA_TRY(cudaMemcpyAsync(F, P->d_F, sizeof(double), cudaMemcpyDeviceToHost, s));
        sync = true;
    }
    if (sync) {
        GRAPE_CUDA_TRY(cudaStreamSynchronize(s));
        return grape_problem_status(P);
    }
    return GRAPE_OK;
}

namespace {

grape_status filter_args(int32_t N, int32_t M, int32_t R, double Dt, double dt, const double *omega0,
                         FilterArgs *a) {
    if (N < 1 || M < 1) return fail(GRAPE_EINVAL, "filter: n_steps and n_sub must be >= 1");
    if (R < 1 || R > GRAPE_MAXR) return fail(GRAPE_EINVAL, "filter: n_controls must be in [1, 8]");
    if (!(Dt > 0.0) || !(dt > 0.0) || !std::isfinite(Dt) || !std::isfinite(dt))
        return fail(GRAPE_EINVAL, "filter: Dt and dt must be positive and finite");
    if (!omega0) return fail(GRAPE_EINVAL, "filter: omega0 is NULL");
    std::memset(a, 0, sizeof(*a));
    a->N = N;
    a->M = M;
    a->R = R;
    a->Dt = Dt;
    a->dt = dt;
    for (int k = 0; k < R; ++k) {
        if (!(omega0[k] > 0.0) || !std::isfinite(omega0[k]))
            return fail(GRAPE_EINVAL, "filter: omega0 must be positive and finite");
        a->w0[k] = omega0[k];
    }
    return GRAPE_OK;
}

grape_status filter_call(int32_t N, int32_t M, int32_t R, double Dt, double dt, const double *omega0,
                         const double *in, double *out, bool adjoint, void *stream) {
    FilterArgs a;
    grape_status st = filter_args(N, M, R, Dt, dt, omega0, &a);
    if (st != GRAPE_OK) return st;
    if (!in || !out) return fail(GRAPE_EINVAL, "filter: input and output must be device memory");
    int dev = 0;
    GRAPE_CUDA_TRY(cudaGetDevice(&dev));
    if ((st = require_device_ptr(in, dev, "filter input")) != GRAPE_OK) return st;
    if ((st = require_device_ptr(out, dev, "filter output")) != GRAPE_OK) return st;
    a.in = in;
    a.out = out;
    GRAPE_CUDA_TRY(grape_launch_filter(a, adjoint, static_cast<cudaStream_t>(stream)));
    return GRAPE_OK;
}

}  // namespace

grape_status grape_filter_apply(int32_t n_steps, int32_t n_sub, int32_t n_controls, double Dt, double dt,
                                const double *omega0, const double *u, double *s, void *stream) {
    return filter_call(n_steps, n_sub, n_controls, Dt, dt, omega0, u, s, false, stream);
}

grape_status grape_filter_adjoint(int32_t n_steps, int32_t n_sub, int32_t n_controls, double Dt, double dt,
                                  const double *omega0, const double *g_s, double *g_u, void *stream) {
    return filter_call(n_steps, n_sub, n_controls, Dt, dt, omega0, g_s, g_u, true, stream);
}

grape_status grape_gradient_filtered(grape_problem_t P, int32_t n_steps, const double *omega0,
                                     const double *u, double *F, double *grad, void *stream) {
    if (!P || !u || !F || !grad) return fail(GRAPE_EINVAL, "NULL problem, u, F or grad");
    if (P->R < 1) return fail(GRAPE_EINVAL, "filtered gradient: the problem has no controls");
    DeviceGuard g(P->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    FilterArgs a;
    grape_status st = filter_args(n_steps, P->n_slices, P->R, P->T / n_steps, P->T / P->n_slices, omega0, &a);
    if (st != GRAPE_OK) return st;
    const size_t sub_b = (size_t)P->n_slices * P->R * sizeof(double);
    const size_t step_b = (size_t)n_steps * P->R * sizeof(double);
    if (!P->d_fs) {
        P->d_fs = static_cast<double *>(P->alloc(sub_b));
        P->d_fgs = static_cast<double *>(P->alloc(sub_b));
        if (!P->d_fs || !P->d_fgs) return fail(GRAPE_ENOMEM, "cudaMalloc failed for filtered controls");
    }
    bool u_dev = false, g_dev = false;
    if ((st = locate_ptr(u, P->device, "u", &u_dev)) != GRAPE_OK) return st;
    if ((st = locate_ptr(grad, P->device, "grad", &g_dev)) != GRAPE_OK) return st;
    if ((!u_dev || !g_dev) && P->f_steps < n_steps) {
        P->d_fu = static_cast<double *>(P->alloc(step_b));
        P->d_fgu = static_cast<double *>(P->alloc(step_b));
        if (!P->d_fu || !P->d_fgu) return fail(GRAPE_ENOMEM, "cudaMalloc failed for staged controls");
        P->f_steps = n_steps;
    }
    if (!u_dev) GRAPE_CUDA_TRY(cudaMemcpyAsync(P->d_fu, u, step_b, cudaMemcpyHostToDevice, s));
    a.in = u_dev ? u : P->d_fu;
    a.out = P->d_fs;
    GRAPE_CUDA_TRY(grape_launch_filter(a, false, s));
    if ((st = grape_gradient(P, P->d_fs, F, P->d_fgs, stream)) != GRAPE_OK) return st;
    a.in = P->d_fgs;
    a.out = g_dev ? grad : P->d_fgu;
    GRAPE_CUDA_TRY(grape_launch_filter(a, true, s));
    if (!g_dev) {
        GRAPE_CUDA_TRY(cudaMemcpyAsync(grad, P->d_fgu, step_b, cudaMemcpyDeviceToHost, s));
        GRAPE_CUDA_TRY(cudaStreamSynchronize(s));
    }
    return GRAPE_OK;
}

grape_status grape_gradient(grape_problem_t P, const double *u, double *F, double *grad,
                            void *stream) {
    if (!P || !F || (!grad && P->R > 0)) return fail(GRAPE_EINVAL, "NULL problem, F or grad");
    DeviceGuard g(P->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    grape_status st;
    bool f_dev = false, g_dev = false;
    if ((st = locate_ptr(F, P->device, "F", &f_dev)) != GRAPE_OK) return st;
    if ((st = locate_ptr(grad, P->device, "grad", &g_dev)) != GRAPE_OK) return st;
    if ((st = plan_gradient(P)) != GRAPE_OK) return st;
    const double *ud;
    if ((st = stage_inputs(P, u, &ud, s)) != GRAPE_OK) return st;
    GradScratch S;
    S.Y = P->d_Y;
    S.K = P->d_K;
    S.ckpt = P->d_ckpt;
    S.x = P->d_x;
    S.mu = P->d_mu;
    S.seg = P->seg;
    S.nseg = P->nseg;
    S.ev = P->ev;
    S.part = P->d_part;
    bool overlap = true;
    if (const char *env = std::getenv("GRAPE_TRACE_OVERLAP")) overlap = std::atoi(env) != 0;
    S.s2 = overlap ? P->s2 : nullptr;
    if (S.s2 && concurrent_sweeps(P, P->nseg)) {
        S.s3 = P->s3;
        S.fork3 = P->ev_fork3;
        S.evF = P->evF;
    }
    // the sweeps run on the problem's high-priority streams, ordered after and
    // before the caller's stream; the traces on its low-priority stream
    GRAPE_CUDA_TRY(cudaEventRecord(P->ev_fork, s));
    GRAPE_CUDA_TRY(cudaStreamWaitEvent(P->s1, P->ev_fork, 0));
    if ((st = run_gradient(P, ud, f_dev ? F : P->d_F, g_dev ? grad : P->d_G, P->s1, S)) != GRAPE_OK)
        return st;
    GRAPE_CUDA_TRY(cudaEventRecord(P->ev_join, P->s1));
    GRAPE_CUDA_TRY(cudaStreamWaitEvent(s, P->ev_join, 0));
    bool sync = false;
    if (!f_dev) {
        GRAPE_CUDA_TRY(cudaMemcpyAsync(F, P->d_F, sizeof(double), cudaMemcpyDeviceToHost, s));
        sync = true;
    }
    if (grad && !g_dev && P->R > 0) {
        GRAPE_CUDA_TRY(cudaMemcpyAsync(grad, P->d_G, (size_t)P->n_slices * P->R * sizeof(double),
                                       cudaMemcpyDeviceToHost, s));
        sync = true;
    }
    if (sync) {
        GRAPE_CUDA_TRY(cudaStreamSynchronize(s));
        return grape_problem_status(P);
    }
    return GRAPE_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// grape_gradient_static: the gradient without any device allocation.
//
// For callers that cannot allocate device memory at the time they need a
// gradient - code running under a custom or pool allocator that owns all of
// the device memory, callbacks and host functions where cudaMalloc may not be
// called, or real-time loops that must not block on the allocator.  The
// problem tables are created beforehand by grape_problem_create; every buffer
// the gradient needs beyond its inputs and outputs (RK stage storage of the
// forward and adjoint sweeps, checkpoints, the propagated and adjoint states,
// the partial traces) comes from the file-scope array below instead of
// cudaMalloc.
namespace {

constexpr size_t kStaticScratchBytes = size_t(64) << 20;   // 64 MiB per device
constexpr int kMaxDevices = 64;

// Device memory held by every GPU that loads this library, until exit.
static __device__ __align__(256) unsigned char g_static_scratch[kStaticScratchBytes];

// Device address of g_static_scratch per device.  In host code the symbol
// name is only a host-side stand-in, never a device address, so it goes
// through cudaGetSymbolAddress once per device, with that device current.
// That lookup also loads the module that holds the array (modules load
// lazily), which is when the 64 MiB are committed on the device: it runs in
// grape_problem_create, which allocates anyway, so that the static entry
// point itself only reads the cached address.
struct StaticScratch {
    std::once_flag once;
    void *ptr = nullptr;
    cudaError_t err = cudaErrorNotReady;
};
StaticScratch g_static[kMaxDevices];

size_t align256(size_t n) { return (n + 255) & ~size_t(255); }

}  // namespace

// with device `dev` current
static void static_scratch_setup(int dev) {
    if (dev < 0 || dev >= kMaxDevices) return;
    StaticScratch &sl = g_static[dev];
    std::call_once(sl.once, [&] {
        void *ptr = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess) cudaGetLastError();
        sl.err = (e == cudaSuccess && !ptr) ? cudaErrorInvalidSymbol : e;
        sl.ptr = (sl.err == cudaSuccess) ? ptr : nullptr;
    });
}

extern "C" {

grape_status grape_gradient_static(grape_problem_t P, const double *u, double *F, double *grad,
                                   void *stream) {
    if (!P || !u || !F || (!grad && P->R > 0)) return fail(GRAPE_EINVAL, "NULL problem, u, F or grad");
    if (P->device < 0 || P->device >= kMaxDevices) return fail(GRAPE_EINVAL, "device index too large");
    DeviceGuard g(P->device);
    grape_status st;
    if ((st = require_device_ptr(u, P->device, "u")) != GRAPE_OK) return st;
    if ((st = require_device_ptr(F, P->device, "F")) != GRAPE_OK) return st;
    if (P->R > 0 && (st = require_device_ptr(grad, P->device, "grad")) != GRAPE_OK) return st;
    if (P->penalty)
        return fail(GRAPE_EINVAL, "grape_gradient_static does not evaluate the running-cost penalty");
    static_scratch_setup(P->device);   // done by grape_problem_create; a no-op here
    if (g_static[P->device].err != cudaSuccess)
        return fail(GRAPE_ECUDA, std::string("cudaGetSymbolAddress(static scratch): ") +
                                     cudaGetErrorString(g_static[P->device].err));
    unsigned char *base = static_cast<unsigned char *>(g_static[P->device].ptr);

    // scratch plan: propagated state, adjoint state, stage storage of one
    // segment (forward and adjoint), the segment's partial traces and, with
    // several segments, the checkpoints
    const bool exact = (P->mode == GRAPE_GRAD_EXACT);
    const int nsplit = std::max(1, P->trace.nsplit);
    const size_t mat = align256(P->d2 * P->ns * sizeof(double2));
    auto per_seg = [&](long long sg) { return align256(stage_bytes(P, sg)); };
    auto part_bytes = [&](long long sg) {
        return nsplit > 1 ? align256((size_t)sg * nsplit * std::max(P->R, 1) * sizeof(double)) : 0;
    };
    auto need = [&](long long sg) {
        const long long ns = (P->n_slices + sg - 1) / sg;
        return 2 * mat + 2 * per_seg(sg) + part_bytes(sg) + (ns > 1 ? (size_t)(ns + 1) * mat : 0);
    };
    // the longest segment that fits (fewest launches); the need is not
    // monotonic in the length (stage storage grows, checkpoints shrink), so
    // every length is tried
    long long seg = 0;
    size_t least = SIZE_MAX;
    for (long long sg = P->n_slices; sg >= 1; --sg) {
        const size_t nb = need(sg);
        least = std::min(least, nb);
        if (nb <= kStaticScratchBytes) { seg = sg; break; }
    }
    if (seg == 0)
        return fail(GRAPE_EINVAL, "problem needs at least " + std::to_string(least) +
                                      " bytes of scratch with every checkpoint segment length; "
                                      "the static scratch holds " + std::to_string(kStaticScratchBytes));
    const int nseg = (int)((P->n_slices + seg - 1) / seg);
    double2 *x = reinterpret_cast<double2 *>(base);
    double2 *mu = reinterpret_cast<double2 *>(base + mat);
    double2 *Y = reinterpret_cast<double2 *>(base + 2 * mat);
    double2 *K = reinterpret_cast<double2 *>(base + 2 * mat + per_seg(seg));
    double *part = reinterpret_cast<double *>(base + 2 * mat + 2 * per_seg(seg));
    double2 *ckpt = reinterpret_cast<double2 *>(base + 2 * mat + 2 * per_seg(seg) + part_bytes(seg));

    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const long long nsub = (long long)P->n_slices * P->n_rk;
    const size_t m = P->d2 * P->ns;
    PropArgs f = base_args(P, 0, u);
    f.sub_begin = 0;
    f.sub_end = nsub;
    f.x_in = P->d_rho0;
    f.x_out = x;
    if (nseg == 1) {
        if (exact) f.stage_store = Y;
        else { f.bound_store = Y; f.bound_step = P->n_rk; }
    } else {
        f.bound_store = ckpt;
        f.bound_step = seg * P->n_rk;
    }
    GRAPE_CUDA_TRY(k_prop(P, f, s));
    GRAPE_CUDA_TRY(k_cost(P, x, F, s));
    GRAPE_CUDA_TRY(cudaMemcpyAsync(mu, P->d_sigma, m * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    for (int gi = nseg - 1; gi >= 0; --gi) {
        const long long j0 = (long long)gi * seg;
        const long long j1 = std::min<long long>(P->n_slices, j0 + seg);
        if (nseg > 1) {
            PropArgs r = base_args(P, 0, u);
            r.sub_begin = j0 * P->n_rk;
            r.sub_end = j1 * P->n_rk;
            r.x_in = ckpt + (size_t)gi * m;   // the kernel writes checkpoints back to back
            r.x_out = x;
            if (exact) r.stage_store = Y;
            else { r.bound_store = Y; r.bound_step = P->n_rk; }
            GRAPE_CUDA_TRY(k_prop(P, r, s));
        }
        PropArgs b = base_args(P, 1, u);
        b.sub_begin = j0 * P->n_rk;
        b.sub_end = j1 * P->n_rk;
        b.reverse = 1;
        b.x_in = mu;
        b.x_out = mu;
        if (exact) b.stage_store = K;
        else { b.bound_store = K; b.bound_step = P->n_rk; }
        GRAPE_CUDA_TRY(k_prop(P, b, s));
        if (P->R == 0) continue;
        // the problem's own split count, so that the traces are summed in
        // the same order as in grape_gradient (identical bits)
        TraceArgs t = P->trace;
        t.nsplit = nsplit;
        t.part = nsplit > 1 ? part : nullptr;
        t.n_rows = (int)(j1 - j0);
        t.G = grad + (size_t)j0 * P->R;
        if (exact) {
            t.K = K;
            t.Y = Y;
            t.npairs = (long long)P->n_rk * 4 * P->ns;
            t.weight = 1.0;
        } else {
            t.K = K + m;
            t.Y = Y + m;
            t.npairs = P->ns;
            t.weight = P->T / P->n_slices;
        }
        GRAPE_CUDA_TRY(k_trace(P, t, s));
        if (nsplit > 1)
            GRAPE_CUDA_TRY(P->prec == GRAPE_PREC_FP64 ? grape_launch_trace_finish_f64(t, s)
                                                      : grape_launch_trace_finish_df(t, s));
    }
    return GRAPE_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batched gradients: many problems of different sizes in one graph launch.
struct grape_batch {
    int device = 0;
    std::vector<grape_problem *> probs;
    int n_lanes = 0;
    std::vector<cudaStream_t> lanes;
    std::vector<cudaEvent_t> lane_done;
    // per lane, for concurrent sweeps: the adjoint's and the traces' streams
    // and the events that order them (kMaxChunks + 2 + kMaxChunks + 1 each)
    std::vector<cudaStream_t> lane_adj, lane_tr;
    std::vector<std::vector<cudaEvent_t>> lane_ev;
    cudaEvent_t fork = nullptr, ev_in = nullptr, ev_out = nullptr;
    cudaStream_t cap = nullptr;                // the graph is captured and launched here
    std::vector<std::vector<int>> items;       // problem indices per lane, run in order
    std::vector<GradScratch> scratch;          // per problem (pointers into its lane's buffers)
    std::vector<void *> allocs;
    size_t bytes = 0;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    std::vector<const void *> key;             // pointers the graph was captured with
    std::vector<int2> own_tile;                // (width, threads) before tuning; x = 0: unchanged
    std::vector<double> copies;                // per problem: copies of it resident at once
    ~grape_batch() {
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        for (auto e : lane_done) cudaEventDestroy(e);
        for (auto &v : lane_ev)
            for (auto e : v)
                if (e) cudaEventDestroy(e);
        for (auto l : lane_adj) if (l) cudaStreamDestroy(l);
        for (auto l : lane_tr) if (l) cudaStreamDestroy(l);
        if (fork) cudaEventDestroy(fork);
        if (ev_in) cudaEventDestroy(ev_in);
        if (ev_out) cudaEventDestroy(ev_out);
        if (cap) cudaStreamDestroy(cap);
        for (auto l : lanes) cudaStreamDestroy(l);
        for (void *p : allocs) cudaFree(p);
    }
};

namespace {

// Clusters of the problem's current tile that can be resident at once.
int resident_clusters(const grape_problem *P) {
    int clusters = 0;
    const cudaError_t e =
        P->prec == GRAPE_PREC_FP64
            ? grape_max_active_clusters_f64(P->threads, P->variant, P->smem, P->ncl, P->ncl * P->ns, &clusters)
            : grape_max_active_clusters_df(P->threads, P->variant, P->smem, P->ncl, P->ncl * P->ns, &clusters);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return 1;
    }
    return std::max(1, clusters);
}

// Tile autotuner.  Problems are grouped into buckets of d (32 wide).  For
// each bucket the largest problem stands in for the rest: for every tile
// (cluster width x threads per CTA) that fits it, a forward propagation of
// a few slices runs as C concurrent copies, C = the copies whose clusters
// can be resident at once (at most kMaxCopies), and the tile with the most
// slices per second over all copies wins.  It is then set on every problem
// of the bucket it fits (results do not depend on the tile).
constexpr int kMaxCopies = 64;
constexpr int kProbeSlices = 32;

grape_status tune_batch(grape_batch *B) {
    const int n = (int)B->probs.size();
    B->own_tile.assign(n, make_int2(0, 0));
    B->copies.assign(n, 1.0);
    std::map<int, std::vector<int>> buckets;
    for (int i = 0; i < n; ++i)
        if (!B->probs[i]->grid) buckets[(B->probs[i]->d - 1) / 32].push_back(i);
    if (buckets.empty()) return GRAPE_OK;
    size_t out_bytes = 16, u_bytes = 16;
    for (auto &kv : buckets)
        for (int i : kv.second) {
            const grape_problem *P = B->probs[i];
            out_bytes = std::max(out_bytes, (size_t)kMaxCopies * P->ns * P->d2 * sizeof(double2));
            u_bytes = std::max(u_bytes, (size_t)kProbeSlices * std::max(P->R, 1) * sizeof(double));
        }
    void *out = nullptr, *u = nullptr;
    std::vector<cudaStream_t> ss(kMaxCopies, nullptr);
    std::vector<cudaEvent_t> done(kMaxCopies, nullptr);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    auto cleanup = [&] {
        for (auto x : ss) if (x) cudaStreamDestroy(x);
        for (auto x : done) if (x) cudaEventDestroy(x);
        if (e0) cudaEventDestroy(e0);
        if (e1) cudaEventDestroy(e1);
        if (out) cudaFree(out);
        if (u) cudaFree(u);
    };
    if (cudaMalloc(&out, out_bytes) != cudaSuccess || cudaMalloc(&u, u_bytes) != cudaSuccess ||
        cudaMemset(u, 0, u_bytes) != cudaSuccess || cudaStreamSynchronize(cudaStreamLegacy) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        cleanup();
        return fail(GRAPE_ENOMEM, "tile tuner: probe buffers");
    }
    for (int k = 0; k < kMaxCopies; ++k)
        if (cudaStreamCreateWithFlags(&ss[k], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&done[k], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            cleanup();
            return fail(GRAPE_ECUDA, "tile tuner: streams");
        }
    // C copies of P's first kProbeSlices slices; milliseconds of the wave
    auto probe = [&](grape_problem *P, int C, float *ms) -> grape_status {
        PropArgs a = base_args(P, 0, static_cast<const double *>(u));
        a.sub_begin = 0;
        a.sub_end = (long long)std::min(kProbeSlices, P->n_slices) * P->n_rk;
        a.x_in = P->d_rho0;
        GRAPE_CUDA_TRY(cudaEventRecord(e0, ss[0]));
        for (int k = 0; k < C; ++k) {
            if (k) GRAPE_CUDA_TRY(cudaStreamWaitEvent(ss[k], e0, 0));
            a.x_out = static_cast<double2 *>(out) + (size_t)k * P->ns * P->d2;
            GRAPE_CUDA_TRY(k_prop(P, a, ss[k]));
            GRAPE_CUDA_TRY(cudaEventRecord(done[k], ss[k]));
            GRAPE_CUDA_TRY(cudaStreamWaitEvent(ss[0], done[k], 0));
        }
        GRAPE_CUDA_TRY(cudaEventRecord(e1, ss[0]));
        GRAPE_CUDA_TRY(cudaEventSynchronize(e1));
        GRAPE_CUDA_TRY(cudaEventElapsedTime(ms, e0, e1));
        return GRAPE_OK;
    };
    static const int kThreads[3] = {128, 256, 512};
    grape_status st = GRAPE_OK;
    for (auto &kv : buckets) {
        std::vector<int> &idx = kv.second;
        int rep = idx[0];
        for (int i : idx) {
            const grape_problem *a = B->probs[i], *b = B->probs[rep];
            if (a->d > b->d || (a->d == b->d && a->ns > b->ns)) rep = i;
        }
        grape_problem *R = B->probs[rep];
        const int2 own = make_int2(R->ncl, R->threads);
        double best = -1.0;
        int2 tile = own;
        for (int w = 1; w <= 16 && st == GRAPE_OK; w *= 2)
            for (int t : kThreads) {
                const grape_status ps = grape_problem_set_tile(R, w, t);
                if (ps == GRAPE_EINVAL) continue;
                if (ps != GRAPE_OK) { st = ps; break; }
                const int C = std::max(1, std::min(kMaxCopies, resident_clusters(R) / R->ns));
                float ms = 0.0f, ms2 = 0.0f;
                if ((st = probe(R, C, &ms)) != GRAPE_OK || (st = probe(R, C, &ms2)) != GRAPE_OK) break;
                const double rate = C / (double)std::max(1e-3f, std::min(ms, ms2));
                if (std::getenv("GRAPE_TUNE_LOG"))
                    std::fprintf(stderr, "tile d=%d states=%d cluster=%d threads=%d copies=%d ms=%.3f rate=%.1f\n",
                                 R->d, R->ns, w, t, C, std::min(ms, ms2), rate);
                if (rate > best) { best = rate; tile = make_int2(w, t); }
            }
        if (st == GRAPE_OK) st = grape_problem_set_tile(R, own.x, own.y);   // back before the sweep below
        if (st != GRAPE_OK) break;
        for (int i : idx) {
            grape_problem *P = B->probs[i];
            const int2 mine = make_int2(P->ncl, P->threads);
            if (tile.x == mine.x && tile.y == mine.y) {
                B->copies[i] = std::max(1, std::min(kMaxCopies, resident_clusters(P) / P->ns));
                continue;
            }
            const grape_status ps = grape_problem_set_tile(P, tile.x, tile.y);
            if (ps == GRAPE_OK) B->own_tile[i] = mine;
            else if (ps != GRAPE_EINVAL) { st = ps; break; }
            B->copies[i] = std::max(1, std::min(kMaxCopies, resident_clusters(P) / P->ns));
        }
        if (st != GRAPE_OK) break;
    }
    cudaDeviceSynchronize();
    cleanup();
    return st;
}

void restore_tiles(grape_batch *B) {
    for (size_t i = 0; i < B->own_tile.size(); ++i)
        if (B->own_tile[i].x > 0) grape_problem_set_tile(B->probs[i], B->own_tile[i].x, B->own_tile[i].y);
}

// rough device time of one gradient, for the longest-first lane assignment
double gradient_cost(const grape_problem *P) {
    const double per_cta = (double)P->cu > 0 ? (double)P->cu : (double)P->chunk;
    const double stage = 1.0 + per_cta * 0.006;   // microseconds
    return 3.0 * P->n_slices * P->n_rk * 4.0 * stage;
}

}  // namespace

extern "C" {

grape_status grape_batch_create(grape_problem_t *problems, int32_t n, int32_t n_lanes,
                                grape_batch_t *out) {
    if (!problems || n <= 0 || !out) return fail(GRAPE_EINVAL, "NULL problems/out or n <= 0");
    *out = nullptr;
    const int dev = problems[0] ? problems[0]->device : 0;
    for (int i = 0; i < n; ++i) {
        if (!problems[i]) return fail(GRAPE_EINVAL, "NULL problem in batch");
        if (problems[i]->device != dev) return fail(GRAPE_EINVAL, "batch problems on different devices");
        for (int k = 0; k < i; ++k)
            if (problems[k] == problems[i]) return fail(GRAPE_EINVAL, "a problem appears twice in the batch");
    }
    DeviceGuard g(dev);
    grape_batch *B = new grape_batch();
    auto bail = [&](grape_status s) { restore_tiles(B); delete B; return s; };
    B->device = dev;
    B->probs.assign(problems, problems + n);
    bool tune = true;
    if (const char *env = std::getenv("GRAPE_BATCH_TUNE")) tune = std::atoi(env) != 0;
    if (tune) {
        const grape_status st = tune_batch(B);
        if (st != GRAPE_OK) return bail(st);
    } else {
        B->own_tile.assign(n, make_int2(0, 0));
        B->copies.assign(n, 1.0);
        for (int i = 0; i < n; ++i)
            if (!B->probs[i]->grid)
                B->copies[i] = std::max(1, std::min(kMaxCopies, resident_clusters(B->probs[i]) / B->probs[i]->ns));
    }
    // lanes: as many as problems of the mix can run at once (work-weighted
    // mean of the resident copies), at least 8
    int lanes = n_lanes;
    if (lanes <= 0) {
        double wsum = 0.0, csum = 0.0;
        for (int i = 0; i < n; ++i) {
            const double c = gradient_cost(B->probs[i]);
            wsum += c;
            csum += c * B->copies[i];
        }
        lanes = std::max(8, (int)std::lround(wsum > 0.0 ? csum / wsum : 8.0));
        lanes = std::min(lanes, 128);
    }
    B->n_lanes = std::max(1, std::min<int>(lanes, n));
    // longest-first assignment to the least loaded lane
    std::vector<int> order(n);
    for (int i = 0; i < n; ++i) order[i] = i;
    std::sort(order.begin(), order.end(), [&](int a, int b) {
        return gradient_cost(B->probs[a]) > gradient_cost(B->probs[b]);
    });
    B->items.assign(B->n_lanes, {});
    std::vector<double> load(B->n_lanes, 0.0);
    for (int i : order) {
        const int l = (int)(std::min_element(load.begin(), load.end()) - load.begin());
        B->items[l].push_back(i);
        load[l] += gradient_cost(B->probs[i]);
    }
    // per-lane scratch, shared by the lane's problems (they run one after another)
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(GRAPE_ECUDA, "cudaMemGetInfo failed"));
    }
    double frac = 0.6;
    if (const char *env = std::getenv("GRAPE_MEM_FRACTION")) {
        const double v = std::atof(env);
        if (v > 0.0 && v <= 0.95) frac = v;
    }
    const size_t lane_budget = (size_t)(frac * (double)free_b) / B->n_lanes;
    B->scratch.assign(n, GradScratch{});
    for (int l = 0; l < B->n_lanes; ++l) {
        size_t ys = 0, cs = 0, ms = 16;
        std::vector<long long> segs;
        for (int i : B->items[l]) {
            grape_problem *P = B->probs[i];
            const size_t mat = P->d2 * sizeof(double2) * P->ns;
            long long seg = P->ckpt_stride > 0 ? std::min<long long>(P->ckpt_stride, P->n_slices)
                                               : seg_for_budget(P, lane_budget > 2 * mat ? lane_budget - 2 * mat : 0);
            if (seg_bytes(P, seg) + 2 * mat > lane_budget && P->ckpt_stride <= 0)
                return bail(fail(GRAPE_ENOMEM, "batch problem does not fit its lane's memory budget"));
            segs.push_back(seg);
            ys = std::max(ys, stage_bytes(P, seg));
            cs = std::max(cs, ckpt_bytes(P, seg));
            ms = std::max(ms, mat);
        }
        auto take = [&](size_t nbytes) -> double2 * {
            void *p = nullptr;
            if (cudaMalloc(&p, std::max<size_t>(nbytes, 16)) != cudaSuccess) {
                cudaGetLastError();
                return nullptr;
            }
            B->allocs.push_back(p);
            B->bytes += nbytes;
            return static_cast<double2 *>(p);
        };
        double2 *Y = take(ys), *K = take(ys), *C = cs ? take(cs) : nullptr, *X = take(ms), *M = take(ms);
        if (!Y || !K || (cs && !C) || !X || !M) return bail(fail(GRAPE_ENOMEM, "cudaMalloc failed for batch scratch"));
        for (size_t t = 0; t < B->items[l].size(); ++t) {
            grape_problem *P = B->probs[B->items[l][t]];
            GradScratch &S = B->scratch[B->items[l][t]];
            S.Y = Y;
            S.K = K;
            S.ckpt = C;
            S.x = X;
            S.mu = M;
            S.seg = (int)segs[t];
            S.nseg = (int)((P->n_slices + segs[t] - 1) / segs[t]);
            S.s2 = nullptr;      // lanes already run concurrently: traces stay on the lane
            S.ev = nullptr;
            S.part = P->d_part;
        }
    }
    B->lanes.resize(B->n_lanes);
    B->lane_done.resize(B->n_lanes);
    for (int l = 0; l < B->n_lanes; ++l) {
        if (cudaStreamCreateWithFlags(&B->lanes[l], cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&B->lane_done[l], cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            return bail(fail(GRAPE_ECUDA, "stream/event creation failed"));
        }
    }
    // concurrent sweeps inside each lane (the problems' forward and adjoint
    // sweeps side by side, as in grape_gradient): GRAPE_BATCH_CONCURRENT=1
    // (measured: the same throughput as one sweep after the other, the batch
    // being bound by SM time, with 22 % more launches; off by default)
    bool lane_conc = false;
    if (const char *env = std::getenv("GRAPE_BATCH_CONCURRENT")) lane_conc = std::atoi(env) != 0;
    if (lane_conc) {
        const int nev = 2 * grape_problem::kMaxChunks + 3;
        B->lane_adj.assign(B->n_lanes, nullptr);
        B->lane_tr.assign(B->n_lanes, nullptr);
        B->lane_ev.assign(B->n_lanes, std::vector<cudaEvent_t>(nev, nullptr));
        for (int l = 0; l < B->n_lanes; ++l) {
            bool ok = cudaStreamCreateWithFlags(&B->lane_adj[l], cudaStreamNonBlocking) == cudaSuccess &&
                      cudaStreamCreateWithFlags(&B->lane_tr[l], cudaStreamNonBlocking) == cudaSuccess;
            for (auto &e : B->lane_ev[l])
                ok = ok && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
            if (!ok) {
                cudaGetLastError();
                return bail(fail(GRAPE_ECUDA, "stream/event creation failed"));
            }
            for (int i : B->items[l]) {
                GradScratch &S = B->scratch[i];
                if (!concurrent_sweeps(B->probs[i], S.nseg)) continue;
                S.s2 = B->lane_tr[l];
                S.s3 = B->lane_adj[l];
                S.ev = B->lane_ev[l].data();                                   // kMaxChunks + 2
                S.evF = B->lane_ev[l].data() + grape_problem::kMaxChunks + 2;  // kMaxChunks
                S.fork3 = B->lane_ev[l][2 * grape_problem::kMaxChunks + 2];
            }
        }
    }
    if (cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&B->ev_in, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&B->ev_out, cudaEventDisableTiming) != cudaSuccess ||
        cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return bail(fail(GRAPE_ECUDA, "event creation failed"));
    }
    *out = B;
    return GRAPE_OK;
}

grape_status grape_batch_destroy(grape_batch_t B) {
    if (!B) return GRAPE_OK;
    DeviceGuard g(B->device);
    restore_tiles(B);
    delete B;
    return GRAPE_OK;
}

grape_status grape_batch_info(grape_batch_t B, int32_t *n_lanes, size_t *scratch_bytes,
                              int32_t *launches) {
    if (!B) return fail(GRAPE_EINVAL, "NULL batch");
    if (n_lanes) *n_lanes = B->n_lanes;
    if (scratch_bytes) *scratch_bytes = B->bytes;
    if (launches) {
        int n = 0;
        for (size_t i = 0; i < B->probs.size(); ++i)
            n += gradient_launch_count(B->probs[i], B->scratch[i].seg, B->scratch[i].nseg,
                                       B->scratch[i].s3 != nullptr);
        *launches = n;
    }
    return GRAPE_OK;
}

grape_status grape_batch_gradient(grape_batch_t B, const double *const *u, double *F,
                                  double *const *grad, void *stream) {
    if (!B || !u || !F || !grad) return fail(GRAPE_EINVAL, "NULL batch, u, F or grad");
    DeviceGuard g(B->device);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int n = (int)B->probs.size();
    std::vector<const void *> key;
    key.reserve(2 * n + 1);
    key.push_back(F);
    for (int i = 0; i < n; ++i) {
        key.push_back(u[i]);
        key.push_back(grad[i]);
    }
    // the graph runs on the batch's own stream, ordered after and before `s`
    auto launch = [&]() -> grape_status {
        GRAPE_CUDA_TRY(cudaEventRecord(B->ev_in, s));
        GRAPE_CUDA_TRY(cudaStreamWaitEvent(B->cap, B->ev_in, 0));
        GRAPE_CUDA_TRY(cudaGraphLaunch(B->exec, B->cap));
        GRAPE_CUDA_TRY(cudaEventRecord(B->ev_out, B->cap));
        GRAPE_CUDA_TRY(cudaStreamWaitEvent(s, B->ev_out, 0));
        return GRAPE_OK;
    };
    if (B->exec && key == B->key) return launch();
    // validate once, outside the capture
    grape_status st = GRAPE_OK;
    const int dev = B->device;
    if ((st = require_device_ptr(F, dev, "batch F")) != GRAPE_OK) return st;
    for (int i = 0; i < n; ++i) {
        if ((st = require_device_ptr(u[i], dev, "batch u")) != GRAPE_OK) return st;
        if (B->probs[i]->R > 0 && (st = require_device_ptr(grad[i], dev, "batch grad")) != GRAPE_OK)
            return st;
    }
    if (B->exec) { cudaGraphExecDestroy(B->exec); B->exec = nullptr; }
    if (B->graph) { cudaGraphDestroy(B->graph); B->graph = nullptr; }
    std::vector<bool> prof(n);
    for (int i = 0; i < n; ++i) { prof[i] = B->probs[i]->profiling; B->probs[i]->profiling = false; }
    GRAPE_CUDA_TRY(cudaStreamBeginCapture(B->cap, cudaStreamCaptureModeRelaxed));
    cudaError_t e = cudaEventRecord(B->fork, B->cap);
    for (int l = 0; l < B->n_lanes && e == cudaSuccess && st == GRAPE_OK; ++l) {
        e = cudaStreamWaitEvent(B->lanes[l], B->fork, 0);
        for (int i : B->items[l]) {
            if (e != cudaSuccess || st != GRAPE_OK) break;
            st = run_gradient(B->probs[i], u[i], F + i, grad[i], B->lanes[l], B->scratch[i]);
        }
        if (e == cudaSuccess && st == GRAPE_OK) e = cudaEventRecord(B->lane_done[l], B->lanes[l]);
        if (e == cudaSuccess && st == GRAPE_OK) e = cudaStreamWaitEvent(B->cap, B->lane_done[l], 0);
    }
    cudaGraph_t graph = nullptr;
    const cudaError_t e2 = cudaStreamEndCapture(B->cap, &graph);
    for (int i = 0; i < n; ++i) B->probs[i]->profiling = prof[i];
    if (st != GRAPE_OK) { if (graph) cudaGraphDestroy(graph); return st; }
    if (e != cudaSuccess || e2 != cudaSuccess) {
        if (graph) cudaGraphDestroy(graph);
        cudaGetLastError();
        return fail(GRAPE_ECUDA, std::string("batch capture: ") + cudaGetErrorString(e != cudaSuccess ? e : e2));
    }
    B->graph = graph;
    GRAPE_CUDA_TRY(cudaGraphInstantiate(&B->exec, graph, 0));
    B->key = key;
    return launch();
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Serving: pulse optimisations (projected L-BFGS on the device) admitted by
// device memory and run with continuous batching.  Every admitted job owns a
// stream; a worker thread launches a job's next iteration (one gradient
// evaluation plus one L-BFGS step) as soon as its previous iteration has
// completed, and admits queued jobs whenever slots and memory free up, so
// iterations of different jobs overlap on the GPU.
struct ServerJob {
    uint64_t ticket = 0;
    grape_problem *P = nullptr;
    grape_opt_params prm{};
    int n = 0;
    std::vector<double> u0;
    double *d_arena = nullptr;        // u, g, ut, dir, S, Y, rho, alpha, F, G
    LbfgsState *d_state = nullptr;
    LbfgsState *h_state = nullptr;    // pinned copy read by the worker
    int pinned_slot = -1;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev = nullptr;
    size_t footprint = 0;             // device bytes the job holds
    size_t reserved = 0;              // budget reserved for it at admission
    LbfgsArgs args{};
    int phase = 0;                    // 0 queued, 1 running, 2 done, 3 failed
    grape_status err = GRAPE_OK;
    std::string err_msg;
    std::vector<double> u_out;
    double F_out = 0.0;
    int evals = 0;
    int sm_demand = 0;                // SMs its clusters take (counted at admission)
    int2 own_tile = {0, 0};           // the problem's tile before admission narrowed it (x = 0: kept)
    std::chrono::steady_clock::time_point t_submit, t_start, t_done;
};

struct grape_server {
    int device = 0;
    int n_sms = 0;                      // streaming multiprocessors of the device
    int sms_in_use = 0;                 // SM demand of the admitted jobs
    bool elastic = true;                // narrow the tiles of jobs admitted next to others
    size_t budget = 0;
    int max_slots = 1;
    cudaMemPool_t pool = nullptr;       // device memory of the admitted jobs
    LbfgsState *pinned = nullptr;       // max_slots status words read by the worker
    std::vector<int> free_pinned;       // worker-owned
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<ServerJob *> queue;
    std::vector<ServerJob *> active;
    std::map<uint64_t, ServerJob *> jobs;
    size_t reserved = 0;
    uint64_t next_ticket = 1;
    bool stop = false;
    std::thread worker;
    ~grape_server() {
        for (auto &kv : jobs) delete kv.second;
    }
};

namespace {

size_t lbfgs_bytes(int n, int m) { return ((size_t)(6 + 2 * m) * n + 2 * m + 2) * sizeof(double); }

// Allocate the job's device state and plan its gradient storage within its
// share of the budget.  Called by the worker thread with the device current.
grape_status start_job(grape_server *S, ServerJob *j) {
    grape_problem *P = j->P;
    const int n = j->n, m = j->prm.lbfgs_m;
    const size_t share = S->budget / std::max(1, S->max_slots);
    const size_t lb = lbfgs_bytes(n, m);
    if (cudaStreamCreateWithFlags(&j->stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&j->ev, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return fail(GRAPE_ECUDA, "job stream creation failed");
    }
    if (P->nseg == 0) {            // stream-ordered gradient storage from the server pool
        P->grad_pool = S->pool;
        P->grad_stream = j->stream;
    }
    grape_status st = plan_gradient(P, share > lb ? share - lb : 1);
    if (st != GRAPE_OK) return st;
    if (cudaMallocFromPoolAsync(reinterpret_cast<void **>(&j->d_arena), lb, S->pool, j->stream) != cudaSuccess ||
        cudaMallocFromPoolAsync(reinterpret_cast<void **>(&j->d_state), sizeof(LbfgsState), S->pool,
                                j->stream) != cudaSuccess || S->free_pinned.empty()) {
        cudaGetLastError();
        return fail(GRAPE_ENOMEM, "job allocation failed");
    }
    j->pinned_slot = S->free_pinned.back();
    S->free_pinned.pop_back();
    j->h_state = S->pinned + j->pinned_slot;
    double *a = j->d_arena;
    LbfgsArgs &A = j->args;
    A.state = j->d_state;
    A.n = n;
    A.m = m;
    A.max_evals = j->prm.max_iters;
    A.u_min = j->prm.u_min;
    A.u_max = j->prm.u_max;
    A.tol = j->prm.tol;
    A.step0 = j->prm.step0;
    A.u = a; a += n;
    A.g = a; a += n;
    A.ut = a; a += n;
    A.dir = a; a += n;
    A.S = a; a += (size_t)m * n;
    A.Y = a; a += (size_t)m * n;
    A.rho = a; a += m;
    A.alpha = a; a += m;
    double *Fd = a; a += 2;
    double *Gd = a;
    A.F = Fd;
    A.G = Gd;
    LbfgsState init{};
    init.step = 1.0;
    init.gamma = 1.0;
    *j->h_state = init;
    GRAPE_CUDA_TRY(cudaMemcpyAsync(j->d_state, j->h_state, sizeof(LbfgsState), cudaMemcpyHostToDevice, j->stream));
    GRAPE_CUDA_TRY(cudaMemcpyAsync(A.ut, j->u0.data(), n * sizeof(double), cudaMemcpyHostToDevice, j->stream));
    GRAPE_CUDA_TRY(cudaStreamSynchronize(j->stream));   // u0 and the pinned state may be reused
    j->footprint = lb + P->grad_bytes;
    return GRAPE_OK;
}

// one iteration: gradient evaluation at ut, then one L-BFGS step
grape_status launch_iteration(ServerJob *j) {
    grape_problem *P = j->P;
    GradScratch S;
    S.Y = P->d_Y;
    S.K = P->d_K;
    S.ckpt = P->d_ckpt;
    S.x = P->d_x;
    S.mu = P->d_mu;
    S.seg = P->seg;
    S.nseg = P->nseg;
    // served jobs overlap each other, not their sweeps or traces: with the
    // concurrent-sweep streams of every job (high-priority adjoints,
    // low-priority traces) the traces starved and continuous batching ran
    // at 0.79x serial (measured, 32 jobs at quarter slice counts)
    S.s2 = nullptr;
    S.ev = P->ev;
    S.part = P->d_part;
    grape_status st = run_gradient(P, j->args.ut, const_cast<double *>(j->args.F),
                                   const_cast<double *>(j->args.G), j->stream, S);
    if (st != GRAPE_OK) return st;
    GRAPE_CUDA_TRY(grape_launch_lbfgs(j->args, j->stream));
    GRAPE_CUDA_TRY(cudaMemcpyAsync(j->h_state, j->d_state, sizeof(LbfgsState), cudaMemcpyDeviceToHost, j->stream));
    GRAPE_CUDA_TRY(cudaEventRecord(j->ev, j->stream));
    return GRAPE_OK;
}

// Releases a finished job's device state without synchronising the device:
// frees are ordered on the job's stream.
void free_job_device(grape_server *S, ServerJob *j) {
    if (j->stream) {
        if (j->d_arena) cudaFreeAsync(j->d_arena, j->stream);
        if (j->d_state) cudaFreeAsync(j->d_state, j->stream);
        if (j->P && j->P->grad_stream == j->stream) j->P->release_grad();
        cudaStreamSynchronize(j->stream);   // this stream only
    }
    if (j->ev) cudaEventDestroy(j->ev);
    if (j->stream) cudaStreamDestroy(j->stream);
    if (j->pinned_slot >= 0) S->free_pinned.push_back(j->pinned_slot);
    j->pinned_slot = -1;
    j->ev = nullptr;
    j->stream = nullptr;
    j->d_arena = nullptr;
    j->d_state = nullptr;
    j->h_state = nullptr;
}

// Between iterations of a narrowed job, with nothing waiting: the widest
// cluster up to its own that the free SMs hold (the GPU drains at the end of
// a burst; the last jobs should not stay narrow on an idle device).
void widen_job_tile(grape_server *S, ServerJob *j) {
    if (j->own_tile.x <= 0) return;
    std::lock_guard<std::mutex> lk(S->mu);
    if (!S->queue.empty()) return;
    const int spare = S->n_sms - S->sms_in_use + j->sm_demand;
    for (int w = j->own_tile.x; w > j->P->ncl; w /= 2) {
        if (j->P->ns * w > spare) continue;
        const int t = (w == j->own_tile.x) ? j->own_tile.y : j->P->threads;
        if (grape_problem_set_tile(j->P, w, t) != GRAPE_OK) continue;
        const int dem = j->P->ns * w;
        S->sms_in_use += dem - j->sm_demand;
        j->sm_demand = dem;
        if (w == j->own_tile.x) j->own_tile = make_int2(0, 0);
        return;
    }
}

void restore_job_tile(ServerJob *j) {
    if (j->own_tile.x > 0) grape_problem_set_tile(j->P, j->own_tile.x, j->own_tile.y);
    j->own_tile = make_int2(0, 0);
}

int job_sm_demand(const grape_server *S, const ServerJob *j) {
    const grape_problem *P = j->P;
    return P->grid ? S->n_sms : std::max(1, P->ns * P->ncl);
}

bool problem_busy(const grape_server *S, const grape_problem *P) {
    for (const ServerJob *a : S->active)
        if (a->P == P) return true;
    return false;
}

void server_loop(grape_server *S) {
    cudaSetDevice(S->device);
    for (;;) {
        std::vector<ServerJob *> admit;
        {
            std::unique_lock<std::mutex> lk(S->mu);
            if (S->active.empty() && S->queue.empty()) {
                if (S->stop) break;
                S->cv_work.wait_for(lk, std::chrono::milliseconds(20));
                continue;
            }
            // admission: FIFO while slots are free and the estimated footprint fits
            while (!S->queue.empty() && (int)(S->active.size() + admit.size()) < S->max_slots) {
                ServerJob *j = S->queue.front();
                if (problem_busy(S, j->P)) break;
                // a grid-kernel job occupies every SM with one cooperative grid: it runs alone
                bool grid_running = false;
                for (const ServerJob *a : S->active) grid_running = grid_running || a->P->grid;
                for (const ServerJob *a : admit) grid_running = grid_running || a->P->grid;
                if (grid_running) break;
                if (j->P->grid && !(S->active.empty() && admit.empty())) break;
                // elastic tiles: a job that shares the GPU runs on the narrowest
                // cluster its state fits (fewer SMs for longer; results unchanged)
                const bool alone = S->active.empty() && admit.empty();
                int2 own = make_int2(0, 0);
                if (S->elastic && S->max_slots > 1 && !j->P->grid && (!alone || S->queue.size() > 1)) {
                    const int2 cur = make_int2(j->P->ncl, j->P->threads);
                    for (int w = 1; w < cur.x; w *= 2)
                        if (grape_problem_set_tile(j->P, w, GRAPE_PROP_THREADS) == GRAPE_OK) {
                            own = cur;
                            break;
                        }
                }
                auto undo = [&] { if (own.x > 0) grape_problem_set_tile(j->P, own.x, own.y); };
                // SM demand: every initial state's cluster needs its own SMs; running
                // more than fits only makes the clusters wait for free GPCs
                const int dem = job_sm_demand(S, j);
                if (S->sms_in_use + dem > S->n_sms && !alone) { undo(); break; }
                const size_t share = S->budget / std::max(1, S->max_slots);
                const size_t need = std::min(share, seg_bytes(j->P, j->P->n_slices) + lbfgs_bytes(j->n, j->prm.lbfgs_m));
                if (S->reserved + need > S->budget && !alone) { undo(); break; }
                S->queue.pop_front();
                S->reserved += need;
                S->sms_in_use += dem;
                j->reserved = need;
                j->sm_demand = dem;
                j->own_tile = own;
                admit.push_back(j);
            }
        }
        for (ServerJob *j : admit) {
            j->t_start = std::chrono::steady_clock::now();
            grape_status st = start_job(S, j);
            if (st == GRAPE_OK) st = launch_iteration(j);
            std::lock_guard<std::mutex> lk(S->mu);
            if (st != GRAPE_OK) {
                j->phase = 3;
                j->err = st;
                j->err_msg = g_last_error;
                S->reserved -= j->reserved;
                S->sms_in_use -= j->sm_demand;
                free_job_device(S, j);
                restore_job_tile(j);
                j->t_done = std::chrono::steady_clock::now();
                S->cv_done.notify_all();
            } else {
                j->phase = 1;
                S->active.push_back(j);
            }
        }
        bool progressed = !admit.empty();
        std::vector<ServerJob *> running;
        {
            std::lock_guard<std::mutex> lk(S->mu);
            running = S->active;
        }
        for (ServerJob *j : running) {
            const cudaError_t q = cudaEventQuery(j->ev);
            if (q == cudaErrorNotReady) continue;
            progressed = true;
            grape_status st = GRAPE_OK;
            if (q != cudaSuccess) {
                cudaGetLastError();
                st = fail(GRAPE_ECUDA, std::string("served job: ") + cudaGetErrorString(q));
            } else if (j->P->grid) {
                st = grape_problem_status(j->P);
            }
            if (st == GRAPE_OK && j->h_state->status == 0) {
                widen_job_tile(S, j);
                st = launch_iteration(j);
                if (st == GRAPE_OK) continue;
            }
            // finished (or failed): copy the result out and release the slot
            if (st == GRAPE_OK) {
                j->u_out.resize(j->n);
                cudaMemcpyAsync(j->u_out.data(), j->args.u, j->n * sizeof(double), cudaMemcpyDeviceToHost,
                                j->stream);
                cudaStreamSynchronize(j->stream);
                j->F_out = -j->h_state->f;
                j->evals = j->h_state->evals;
            }
            free_job_device(S, j);
            restore_job_tile(j);
            std::lock_guard<std::mutex> lk(S->mu);
            j->phase = (st == GRAPE_OK) ? 2 : 3;
            j->err = st;
            if (st != GRAPE_OK) j->err_msg = g_last_error;
            j->t_done = std::chrono::steady_clock::now();
            S->reserved -= j->reserved;
            S->sms_in_use -= j->sm_demand;
            S->active.erase(std::find(S->active.begin(), S->active.end(), j));
            S->cv_done.notify_all();
        }
        if (!progressed) std::this_thread::sleep_for(std::chrono::microseconds(50));
    }
}

}  // namespace

extern "C" {

grape_status grape_server_create(size_t hbm_budget_bytes, int32_t max_slots, grape_server_t *out) {
    if (!out || max_slots < 1) return fail(GRAPE_EINVAL, "NULL output or max_slots < 1");
    *out = nullptr;
    grape_server *S = new grape_server();
    if (cudaGetDevice(&S->device) != cudaSuccess) {
        cudaGetLastError();
        delete S;
        return fail(GRAPE_ECUDA, "no CUDA device");
    }
    if (hbm_budget_bytes == 0) {
        size_t free_b = 0, total_b = 0;
        if (cudaMemGetInfo(&free_b, &total_b) != cudaSuccess) {
            cudaGetLastError();
            delete S;
            return fail(GRAPE_ECUDA, "cudaMemGetInfo failed");
        }
        hbm_budget_bytes = (size_t)(0.6 * (double)free_b);
    }
    S->budget = hbm_budget_bytes;
    S->max_slots = max_slots;
    cudaDeviceGetAttribute(&S->n_sms, cudaDevAttrMultiProcessorCount, S->device);
    if (const char *env = std::getenv("GRAPE_SERVER_ELASTIC")) S->elastic = std::atoi(env) != 0;
    cudaMemPoolProps props = {};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = S->device;
    if (cudaMemPoolCreate(&S->pool, &props) != cudaSuccess ||
        cudaMallocHost(&S->pinned, sizeof(LbfgsState) * max_slots) != cudaSuccess) {
        cudaGetLastError();
        delete S;
        return fail(GRAPE_ECUDA, "server pool creation failed");
    }
    unsigned long long keep = ~0ull;   // freed job memory stays in the pool for the next job
    cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    for (int i = max_slots - 1; i >= 0; --i) S->free_pinned.push_back(i);
    S->worker = std::thread(server_loop, S);
    *out = S;
    return GRAPE_OK;
}

grape_status grape_server_destroy(grape_server_t S) {
    if (!S) return GRAPE_OK;
    {
        std::lock_guard<std::mutex> lk(S->mu);
        S->stop = true;
        // queued jobs are dropped; running jobs finish
        for (ServerJob *j : S->queue) {
            j->phase = 3;
            j->err = GRAPE_EINVAL;
            j->err_msg = "server destroyed";
        }
        S->queue.clear();
    }
    S->cv_work.notify_all();
    if (S->worker.joinable()) S->worker.join();
    {
        DeviceGuard g(S->device);
        cudaDeviceSynchronize();
        if (S->pool) cudaMemPoolDestroy(S->pool);
        if (S->pinned) cudaFreeHost(S->pinned);
    }
    delete S;
    return GRAPE_OK;
}

grape_status grape_submit(grape_server_t S, grape_problem_t P, const double *u0,
                          const grape_opt_params *prm, uint64_t *ticket) {
    if (!S || !P || !u0 || !prm || !ticket) return fail(GRAPE_EINVAL, "NULL argument");
    if (P->device != S->device) return fail(GRAPE_EINVAL, "problem on another device");
    if (P->R < 1) return fail(GRAPE_EINVAL, "problem has no controls");
    if (prm->max_iters < 1 || prm->lbfgs_m < 1 || prm->lbfgs_m > 64 || !(prm->u_max > prm->u_min) ||
        !(prm->step0 > 0.0) || prm->tol < 0.0)
        return fail(GRAPE_EINVAL, "bad optimisation parameters");
    ServerJob *j = new ServerJob();
    j->P = P;
    j->prm = *prm;
    j->n = P->n_slices * P->R;
    j->u0.assign(u0, u0 + j->n);
    for (double &v : j->u0) v = std::min(std::max(v, prm->u_min), prm->u_max);
    j->t_submit = std::chrono::steady_clock::now();
    {
        std::lock_guard<std::mutex> lk(S->mu);
        if (S->stop) {
            delete j;
            return fail(GRAPE_EBUSY, "server is shutting down");
        }
        j->ticket = S->next_ticket++;
        S->jobs[j->ticket] = j;
        S->queue.push_back(j);
        *ticket = j->ticket;
    }
    S->cv_work.notify_all();
    return GRAPE_OK;
}

grape_status grape_poll(grape_server_t S, uint64_t ticket, int64_t timeout_us, double *u_out,
                        double *F_out, grape_job_info *info) {
    if (!S) return fail(GRAPE_EINVAL, "NULL server");
    std::unique_lock<std::mutex> lk(S->mu);
    auto it = S->jobs.find(ticket);
    if (it == S->jobs.end()) return fail(GRAPE_EINVAL, "unknown ticket");
    ServerJob *j = it->second;
    if (j->phase < 2 && timeout_us > 0)
        S->cv_done.wait_for(lk, std::chrono::microseconds(timeout_us), [&] { return j->phase >= 2; });
    if (j->phase < 2) return GRAPE_ENOTREADY;
    if (j->phase == 3) {
        const grape_status e = j->err;
        const std::string msg = j->err_msg;
        S->jobs.erase(it);
        delete j;
        return fail(e, msg.empty() ? "job failed" : msg);
    }
    if (u_out) std::memcpy(u_out, j->u_out.data(), j->n * sizeof(double));
    if (F_out) *F_out = j->F_out;
    if (info) {
        using us = std::chrono::duration<double, std::micro>;
        info->evaluations = j->evals;
        info->queued_us = us(j->t_start - j->t_submit).count();
        info->latency_us = us(j->t_done - j->t_submit).count();
    }
    S->jobs.erase(it);
    delete j;
    return GRAPE_OK;
}

}  // extern "C"
