// grape_lbfgs.cu - one iteration of projected L-BFGS on the device, for the
// serving loop's pulse optimisations.
//
// The optimiser maximises Phi by minimising f = -Phi over the box
// u_min <= u <= u_max (Sec. 2.1 of the paper uses BFGS, Eq. update).  Each
// call consumes the gradient evaluation at the trial point ut (F, G written
// by the gradient kernels), decides whether to accept it (plain decrease of
// f; otherwise the step is halved), stores the curvature pair, and writes the
// next trial point: the two-loop recursion applied to the projected gradient
// q (components zeroed whose variable sits on a bound the gradient pushes
// against), those components zeroed in the direction, the scaled -q instead
// when that is not a descent direction, a step along it and a clamp to the
// box.  One CTA,
// FP64, fixed-order shared-memory reductions: the result is a deterministic
// function of the job's own inputs.
#include "grape_internal.h"

namespace {

constexpr int kThreads = 512;

__device__ double block_sum(double v, double *red) {
    // fixed-order tree reduction over the block
    red[threadIdx.x] = v;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

__device__ double block_max(double v, double *red) {
    red[threadIdx.x] = v;
    __syncthreads();
    for (int w = kThreads / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + w]);
        __syncthreads();
    }
    const double r = red[0];
    __syncthreads();
    return r;
}

__device__ double dot(const double *a, const double *b, int n, double *red) {
    double s = 0.0;
    for (int i = threadIdx.x; i < n; i += kThreads) s = fma(a[i], b[i], s);
    return block_sum(s, red);
}

__global__ void __launch_bounds__(kThreads) lbfgs_kernel(LbfgsArgs p) {
    __shared__ double red[kThreads];
    LbfgsState &st = *p.state;
    const int n = p.n, m = p.m;
    double *u = p.u, *g = p.g, *ut = p.ut, *d = p.dir;
    const double ft = -(*p.F);
    // accept or reject the trial point
    bool accept;
    if (st.evals == 0) {
        accept = true;
    } else {
        accept = ft < st.f;
    }
    if (accept && st.evals > 0) {
        // curvature pair s = ut - u, y = gt - g into the ring slot `head`
        double *s = p.S + (size_t)st.head * n, *y = p.Y + (size_t)st.head * n;
        for (int i = threadIdx.x; i < n; i += kThreads) {
            s[i] = ut[i] - u[i];
            y[i] = -p.G[i] - g[i];
        }
        __syncthreads();
        const double sy = dot(s, y, n, red);
        const double ss = dot(s, s, n, red), yy = dot(y, y, n, red);
        if (threadIdx.x == 0 && sy > 1e-12 * sqrt(ss * yy)) {
            p.rho[st.head] = 1.0 / sy;
            st.gamma = sy / yy;
            st.head = (st.head + 1) % m;
            st.hist = min(st.hist + 1, m);
        }
        __syncthreads();
    }
    if (accept) {
        for (int i = threadIdx.x; i < n; i += kThreads) {
            u[i] = ut[i];
            g[i] = -p.G[i];
        }
        if (threadIdx.x == 0) {
            st.f = ft;
            st.step = 1.0;
            st.accepted += 1;
        }
    } else if (threadIdx.x == 0) {
        st.step *= 0.5;
    }
    if (threadIdx.x == 0) st.evals += 1;
    __syncthreads();
    // projected-gradient norm and stopping rules
    double pg = 0.0;
    for (int i = threadIdx.x; i < n; i += kThreads) {
        const double v = fmin(fmax(u[i] - g[i], p.u_min), p.u_max) - u[i];
        pg = fmax(pg, fabs(v));
    }
    pg = block_max(pg, red);
    if (threadIdx.x == 0) st.pgnorm = pg;
    if (st.evals >= p.max_evals || pg <= p.tol || st.step < 1e-10) {
        if (threadIdx.x == 0) st.status = (st.evals >= p.max_evals) ? 1 : 2;
        return;
    }
    // two-loop recursion d = H q on the projected gradient q
    auto active = [&](int i) {
        return (u[i] <= p.u_min && g[i] > 0.0) || (u[i] >= p.u_max && g[i] < 0.0);
    };
    double qmax = 0.0;
    for (int i = threadIdx.x; i < n; i += kThreads) {
        d[i] = active(i) ? 0.0 : g[i];
        qmax = fmax(qmax, fabs(d[i]));
    }
    qmax = block_max(qmax, red);
    const int h = st.hist;
    for (int t = 0; t < h; ++t) {                    // newest to oldest
        const int slot = (st.head - 1 - t + 2 * m) % m;
        const double a = p.rho[slot] * dot(p.S + (size_t)slot * n, d, n, red);
        if (threadIdx.x == 0) p.alpha[slot] = a;
        for (int i = threadIdx.x; i < n; i += kThreads) d[i] -= a * p.Y[(size_t)slot * n + i];
        __syncthreads();
    }
    const double scale = h > 0 ? st.gamma : (qmax > 0.0 ? p.step0 / qmax : 0.0);
    for (int i = threadIdx.x; i < n; i += kThreads) d[i] *= scale;
    __syncthreads();
    for (int t = h - 1; t >= 0; --t) {               // oldest to newest
        const int slot = (st.head - 1 - t + 2 * m) % m;
        const double b = p.rho[slot] * dot(p.Y + (size_t)slot * n, d, n, red);
        const double a = p.alpha[slot];
        for (int i = threadIdx.x; i < n; i += kThreads) d[i] += (a - b) * p.S[(size_t)slot * n + i];
        __syncthreads();
    }
    // direction -d without the bound components; descent check against q
    double dq = 0.0;
    for (int i = threadIdx.x; i < n; i += kThreads) {
        d[i] = active(i) ? 0.0 : -d[i];
        dq = fma(d[i], active(i) ? 0.0 : g[i], dq);
    }
    dq = block_sum(dq, red);
    const bool descent = dq < 0.0;
    const double step = st.step;
    for (int i = threadIdx.x; i < n; i += kThreads) {
        const double di = descent ? d[i] : (active(i) ? 0.0 : -scale * g[i]);
        ut[i] = fmin(fmax(u[i] + step * di, p.u_min), p.u_max);
    }
}

}  // namespace

cudaError_t grape_launch_lbfgs(const LbfgsArgs &a, cudaStream_t s) {
    lbfgs_kernel<<<1, kThreads, 0, s>>>(a);
    return cudaGetLastError();
}
