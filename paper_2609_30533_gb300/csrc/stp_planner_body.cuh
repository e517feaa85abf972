// Planner kernels of the batch-synchronous space-time Extend iteration
// (Algorithm 1 inside Algorithm 2 "IntervalRoot" and Algorithm 3
// "RootRecycle").
//
// One iteration is a fixed sequence of launches (captured into CUDA graphs by
// the host):
//   k_sample        one thread per worker: direction, group/slot, goal time T
//                   (interval root), Philox draws, conditional query sample
//                   (Eq. conditional-query-time), source-set choice, NN query
//                   registration.
//   k_nn            tile scheduler over (tree set, query tile, node tile):
//                   nodes staged in shared memory, one query per thread,
//                   argmin of the directed metric (Eq. space-time-metric) or the
//                   configuration distance; FP32 keys reduced with a packed
//                   64-bit atomicMin (key, index), FP64 keys by the last CTA of
//                   each query tile (both deterministic, ties to lowest index);
//                   the last CTA of a query tile then steers its queries
//                   (Algorithm 1 / Eq. max-speed-extension), checks the horizon
//                   and writes the edge entries. Virtual-root workers are
//                   steered inside k_sample.
//   k_validate      collision kernel over all extension (and root) checks.
//   k_insert        single CTA: ordered insertion in worker order, virtual-root
//                   materialisation, bridge query registration.
//   k_bridge        tile scheduler: best-ranked admissible vertex of the
//                   opposite start-of-iteration set (arrival time, then rho);
//                   the last CTA of a query tile computes the candidate (U, C),
//                   tests the improvement and emits the bridge edge.
//   k_validate      collision kernel over bridge edges.
//   k_publish       single CTA: lexicographic min of (U, C, worker), incumbent
//                   update, interval repartition or root recycling.
// Every kernel returns at once when the control block says the plan is done.
#pragma once

#include "stp_internal.cuh"

namespace stp {

constexpr int kSampleThreads = 128;
constexpr int kCtaThreads = 1024;

enum WorkerStatus { kSkip = 0, kNN = 1, kVirtual = 2 };


template <typename R>
__device__ __forceinline__ R uni_r(uint32_t x) {
    return (R)(x >> 8) * (R)(1.0 / 16777216.0);
}

template <typename R>
__device__ __forceinline__ R* fnode(const State<R>& S, int i) {
    return S.fx + (size_t)i * kDP;
}
template <typename R>
__device__ __forceinline__ R* bnode(const State<R>& S, int seg, int i) {
    return S.bx + ((size_t)seg * S.cap_s + i) * kDP;
}
template <typename R>
__device__ __forceinline__ size_t bofs(const State<R>& S, int seg, int i) {
    return (size_t)seg * S.cap_s + i;
}

// Node rows (kDP values, 16-byte aligned) moved as 16-byte vectors.
template <typename R>
__device__ __forceinline__ void ld_row(const R* src, R (&v)[kDP]) {
    if constexpr (sizeof(R) == 4) {
        const float4 a = reinterpret_cast<const float4*>(src)[0], b = reinterpret_cast<const float4*>(src)[1];
        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
    } else {
#pragma unroll
        for (int k = 0; k < kDP / 2; ++k) {
            const double2 a = reinterpret_cast<const double2*>(src)[k];
            v[2 * k] = a.x;
            v[2 * k + 1] = a.y;
        }
    }
}
template <typename R>
__device__ __forceinline__ void st_row(R* dst, const R (&v)[kDP]) {
    if constexpr (sizeof(R) == 4) {
        reinterpret_cast<float4*>(dst)[0] = make_float4(v[0], v[1], v[2], v[3]);
        reinterpret_cast<float4*>(dst)[1] = make_float4(v[4], v[5], v[6], v[7]);
    } else {
#pragma unroll
        for (int k = 0; k < kDP / 2; ++k) reinterpret_cast<double2*>(dst)[k] = make_double2(v[2 * k], v[2 * k + 1]);
    }
}
// Configuration distance |b - a| over the first dof coordinates of two rows
// held in registers (unrolled with a predicate, so the rows stay in registers).
template <typename R, int N>
__device__ __forceinline__ R qdist_rows(const R (&a)[N], const R (&b)[N], int dof) {
    static_assert(N >= kMaxDof, "rows hold every configuration coordinate");
    R s = R(0);
#pragma unroll
    for (int j = 0; j < kMaxDof; ++j) {
        if (j < dof) {
            R e = b[j] - a[j];
            s += e * e;
        }
    }
    return rsqrt_r(s);
}

// Goal-grid time k dt as stored in the trees (rounded to the working precision,
// so that slot times, node root times and the incumbent compare consistently).
template <typename R>
__device__ __forceinline__ double grid_t(long long k, double dt) {
    return (double)(R)((double)k * dt);
}

// ---------------------------------------------------------------------------
// Interval-root allocation (Sec. "Interval Root"), double precision, one thread.
// ---------------------------------------------------------------------------
template <typename R>
__device__ void build_windows(const State<R>& S) {
    Ctl* c = S.ctl;
    int nw = 0;
    long long k = c->kmin;
    const long long kmax = c->kmin + c->nk - 1;
    while (k <= kmax) {
        if (!S.gfree[k - c->kmin]) {
            ++k;
            continue;
        }
        long long k0 = k;
        while (k + 1 <= kmax && S.gfree[k + 1 - c->kmin]) ++k;
        double lo = __dsub_rn(__dmul_rn((double)k0, c->dt), __dmul_rn(0.5, c->dt));
        double hi = __dadd_rn(__dmul_rn((double)k, c->dt), __dmul_rn(0.5, c->dt));
        lo = fmax(lo, c->Lg);
        hi = fmin(hi, c->H);
        if (hi > lo) {
            S.win_lo[nw] = lo;
            S.win_hi[nw] = hi;
            ++nw;
        }
        ++k;
    }
    c->n_windows = nw;
}

template <typename R>
__device__ void partition(const State<R>& S, double U) {
    Ctl* c = S.ctl;
    const int N = S.N;
    c->Ubar = fmin(c->H, U);
    c->width = (c->Ubar - c->Lg) / (double)N;
    c->n_pieces = 0;
    for (int g = 0; g < N; ++g) {
        c->g_first[g] = 0;
        c->g_count[g] = 0;
        c->g_meas[g] = 0.0;
    }
    // Total guided measure below Ubar.
    double G = 0.0;
    for (int i = 0; i < c->n_windows; ++i) {
        double a = S.win_lo[i];
        if (a >= c->Ubar) continue;
        double b = fmin(S.win_hi[i], c->Ubar);
        if (b > a) G += b - a;
    }
    if (G <= 0.0) return;
    int np = 0;
    for (int g = 0; g < N; ++g) {
        double mlo = G * (double)g / (double)N;
        double mhi = (g == N - 1) ? G : G * (double)(g + 1) / (double)N;
        c->g_first[g] = np;
        double m0 = 0.0;
        for (int i = 0; i < c->n_windows; ++i) {
            double a = S.win_lo[i];
            if (a >= c->Ubar) continue;
            double b = fmin(S.win_hi[i], c->Ubar);
            if (!(b > a)) continue;
            // Same summation order as G, so the last window ends exactly at G.
            double m1 = m0 + (b - a);
            double x = fmax(mlo, m0), y = fmin(mhi, m1);
            if (y > x && np < S.max_pieces) {
                S.pc_lo[np] = a + (x - m0);
                S.pc_hi[np] = a + (y - m0);
                S.pc_group[np] = g;
                c->g_meas[g] += S.pc_hi[np] - S.pc_lo[np];
                ++np;
            }
            m0 = m1;
        }
        c->g_count[g] = np - c->g_first[g];
    }
    c->n_pieces = np;
}

// Goal time of group g (Sec. Interval Root), in the working precision: the
// guided coin is the integer test m_coin < ceil(p_guided 2^24), equivalent to
// u_coin < p_guided for u = m 2^-24.
template <typename R>
__device__ R sample_goal_time(const State<R>& S, int g, uint32_t m_coin, R u_pos, bool& guided) {
    const Ctl* c = S.ctl;
    const R meas = (R)c->g_meas[g];
    guided = m_coin < S.thr_guided && meas > R(0);
    if (guided) {
        R p = u_pos * meas;
        const int f = c->g_first[g], n = c->g_count[g];
        for (int j = 0; j < n; ++j) {
            const R lo = (R)S.pc_lo[f + j], hi = (R)S.pc_hi[f + j];
            const R len = hi - lo;
            if (p < len || j + 1 == n) return (lo + p) < hi ? (lo + p) : hi;
            p -= len;
        }
    }
    const R width = (R)c->width;
    const R lo = (R)c->Lg + (R)g * width;
    return lo + u_pos * width;
}

// ---------------------------------------------------------------------------
// Learned sampling branch (the method's GPU form: a learned proposal mixed
// with 10 % plain samples). A learned worker (slot-12 coin) draws q_r
// uniformly within +-0.1 of each joint range around waypoint i (slot 13),
// clipped to C, reusing the plain q_r uniforms; in interval root its goal
// time comes from the mixture (component by slot 14, Box-Muller normal from
// slots 15-16) when that time lies in the sampled group's uniform interval.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void learned_q(const Geom<R>& G, const State<R>& S, const uint32_t (&d)[20],
                                          R (&qr)[kMaxDof]) {
    const int i = (int)(((unsigned long long)(d[13] >> 8) * 16ull) >> 24);
    const R* wq = S.prop + 24 + i * kMaxDof;
#pragma unroll
    for (int j = 0; j < kMaxDof; ++j) {
        if (j < G.dof) {
            const R half = R(0.1) * (G.qhi[j] - G.qlo[j]);
            R q = wq[j] + half * (R(2) * uni_r<R>(d[4 + j]) - R(1));
            q = q > G.qlo[j] ? q : G.qlo[j];
            qr[j] = q < G.qhi[j] ? q : G.qhi[j];
        }
    }
}

__device__ __forceinline__ float log_r(float x) { return logf(x); }
__device__ __forceinline__ double log_r(double x) { return log(x); }
__device__ __forceinline__ float cos_r(float x) { return cosf(x); }
__device__ __forceinline__ double cos_r(double x) { return cos(x); }
__device__ __forceinline__ float exp_r(float x) { return expf(x); }
__device__ __forceinline__ double exp_r(double x) { return exp(x); }

template <typename R>
__device__ __forceinline__ R learned_T(const State<R>& S, const uint32_t (&d)[20], int& comp) {
    const R u = uni_r<R>(d[14]);
    int k = 0;
    while (k < 7 && !(u < S.prop[k])) ++k;
    comp = k;
    const R u1 = R(1) - uni_r<R>(d[15]), u2 = uni_r<R>(d[16]);
    const R z = sqrt(R(-2) * log_r(u1)) * cos_r(R(6.283185307179586476925) * u2);
    return S.prop[8 + k] + S.prop[16 + k] * z;
}

// Proposal table from the network output (one thread; same operation order
// as the reference construction).
template <typename R>
__global__ void k_set_proposal(Geom<R> G, State<R> S) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const float* y = S.prop_y;
    R amax = (R)y[0];
    for (int k = 1; k < 8; ++k) amax = (R)y[k] > amax ? (R)y[k] : amax;
    R e[8], tot = R(0);
    for (int k = 0; k < 8; ++k) {
        e[k] = exp_r((R)y[k] - amax);
        tot += e[k];
    }
    R acc = R(0);
    for (int k = 0; k < 8; ++k) {
        acc += e[k];
        S.prop[k] = acc / tot;
    }
    S.prop[7] = R(1);
    const R H = (R)S.H;
    for (int k = 0; k < 8; ++k) {
        S.prop[8 + k] = (R)y[8 + k] * H;
        R s = (R)y[16 + k];
        s = s > R(-7) ? s : R(-7);
        s = s < R(2) ? s : R(2);
        S.prop[16 + k] = exp_r(s) * H;
    }
    // Waypoint offsets are taken from the straight line between the
    // normalised start and goal.
    for (int i = 0; i < 16; ++i) {
        const R f = (R)(i + 1) / R(17);
        for (int j = 0; j < kMaxDof; ++j) {
            R v = R(0);
            if (j < G.dof) {
                const R us = R(2) * (S.qs[j] - G.qlo[j]) / (G.qhi[j] - G.qlo[j]) - R(1);
                const R ug = R(2) * (S.qg[j] - G.qlo[j]) / (G.qhi[j] - G.qlo[j]) - R(1);
                R u = (R)y[24 + 8 * i + j] + ((R(1) - f) * us + f * ug);
                u = u > R(-1) ? u : R(-1);
                u = u < R(1) ? u : R(1);
                v = G.qlo[j] + (u + R(1)) * R(0.5) * (G.qhi[j] - G.qlo[j]);
            }
            S.prop[24 + i * kMaxDof + j] = v;
        }
    }
}

// Training targets [130] of the last extracted path (one thread): tau = U/H,
// the path sampled at t_i = (i+1) U / 17 by linear interpolation in t (the
// segment with t_k <= t_i < t_k+1, clamped to the path), joints normalised to
// [-1, 1] and taken relative to the straight line (1 - f_i) u_s + f_i u_g
// between the path's normalised end states (f_i = (i+1)/17), the time entry
// t_i / H, and d. out[130] = 1 if written, 0 if the problem has no path of at
// least two states.
template <typename R>
__global__ void k_path_targets(Geom<R> G, State<R> S, float* out) {
    if (blockIdx.x != 0 || threadIdx.x != 0) return;
    const int n = *S.path_len;
    out[130] = 0.f;
    if (n < 2) return;
    const R* P = S.path;
    const R U = P[(size_t)(n - 1) * kDP + kDP - 1];
    const R H = (R)S.H;
    for (int i = 0; i < 130; ++i) out[i] = 0.f;
    out[0] = (float)(U / H);
    for (int i = 0; i < 16; ++i) {
        const R ti = (R)(i + 1) * U / R(17);
        int cnt = 0;
        for (int k = 0; k < n; ++k)
            if (P[(size_t)k * kDP + kDP - 1] <= ti) ++cnt;
        int k = cnt - 1;
        k = k < 0 ? 0 : (k > n - 2 ? n - 2 : k);
        const R* a = P + (size_t)k * kDP;
        const R* b = a + kDP;
        const R f = (ti - a[kDP - 1]) / (b[kDP - 1] - a[kDP - 1]);
        const R fi = (R)(i + 1) / R(17);
        const R* e = P + (size_t)(n - 1) * kDP;
        for (int j = 0; j < G.dof; ++j) {
            const R q = a[j] + f * (b[j] - a[j]);
            const R span = G.qhi[j] - G.qlo[j];
            const R us = R(2) * (P[j] - G.qlo[j]) / span - R(1);
            const R ug = R(2) * (e[j] - G.qlo[j]) / span - R(1);
            out[1 + 8 * i + j] = (float)((R(2) * (q - G.qlo[j]) / span - R(1)) - ((R(1) - fi) * us + fi * ug));
        }
        out[1 + 8 * i + 7] = (float)(ti / H);
    }
    out[129] = (float)G.dof;
    out[130] = 1.f;
}

template <typename R>
cudaError_t launch_path_targets(const Geom<R>& G, const State<R>& S, float* out, cudaStream_t st) {
    k_path_targets<R><<<1, 1, 0, st>>>(G, S, out);
    return cudaGetLastError();
}
template cudaError_t launch_path_targets<float>(const Geom<float>&, const State<float>&, float*, cudaStream_t);
template cudaError_t launch_path_targets<double>(const Geom<double>&, const State<double>&, float*, cudaStream_t);

template <typename R>
cudaError_t launch_set_proposal(const Geom<R>& G, const State<R>& S, cudaStream_t st) {
    k_set_proposal<R><<<1, 1, 0, st>>>(G, S);
    return cudaGetLastError();
}
template cudaError_t launch_set_proposal<float>(const Geom<float>&, const State<float>&, cudaStream_t);
template cudaError_t launch_set_proposal<double>(const Geom<double>&, const State<double>&, cudaStream_t);

// ---------------------------------------------------------------------------
// Root recycling (Algorithm 3), one thread.
// ---------------------------------------------------------------------------
template <typename R>
__device__ void install_root(const State<R>& S, int slot, double T, int gen, int iter) {
    R* x = bnode(S, slot, 0);
    for (int j = 0; j < kDP; ++j) x[j] = R(0);
    for (int j = 0; j < kMaxDof; ++j) x[j] = S.qg[j];
    x[kDP - 1] = (R)T;
    size_t o = bofs(S, slot, 0);
    S.bpar[o] = -1;
    S.bcost[o] = R(0);
    S.btroot[o] = (R)T;
    S.btree[o] = gen;
    S.biter[o] = iter;
    S.ctl->n_s[slot] = 1;
}

template <typename R>
__device__ void recycle(const State<R>& S, double U, int* donors, long long* held) {
    Ctl* c = S.ctl;
    long long kU = c->kmin;
    while (grid_t<R>(kU, c->dt) < U) ++kU;
    int m = 0, nh = 0;
    for (int i = 0; i < S.N; ++i) {
        if (c->slot_has[i] && c->slot_T[i] >= U) c->slot_active[i] = 0;
        if (!c->slot_has[i] || c->slot_T[i] > U) donors[m++] = i;
        if (c->slot_has[i] && c->slot_active[i]) held[nh++] = c->slot_k[i];
    }
    const long long KU = kU - c->kmin;
    for (int j = 0; j < m && KU > 0; ++j) {
        long long target = c->kmin + ((2LL * j + 1) * KU) / (2LL * m);
        long long found = -1;
        for (long long o = 0; o < KU && found < 0; ++o) {
            for (int side = 0; side < (o == 0 ? 1 : 2); ++side) {
                long long k = side == 0 ? target - o : target + o;
                if (k < c->kmin || k >= kU) continue;
                if (k - c->kmin >= c->nk || !S.gfree[k - c->kmin]) continue;
                bool h = false;
                for (int q = 0; q < nh; ++q) h = h || (held[q] == k);
                if (h) continue;
                found = k;
                break;
            }
        }
        if (found < 0) continue;
        int i = donors[j];
        c->slot_has[i] = 1;
        c->slot_active[i] = 1;
        c->slot_k[i] = found;
        c->slot_T[i] = grid_t<R>(found, c->dt);
        c->slot_gen[i] += 1;
        held[nh++] = found;
        install_root(S, i, c->slot_T[i], c->slot_gen[i], c->iter);
    }
}

// ---------------------------------------------------------------------------
// Reset: fresh trees and allocation for a new plan.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void reset_body(const State<R>& S, int max_iters) {
    Ctl* c = S.ctl;
    const int t = threadIdx.x;
    if (t == 0) {
        c->iter = 0;
        c->err = 0;
        c->n_f = 1;
        c->snap_f = 1;
        c->n_trees = 0;
        c->U = __longlong_as_double(0x7ff0000000000000LL);
        c->C = c->U;
        c->inc_f = c->inc_s = c->inc_b = -1;
        c->first_iter = -1;
        c->max_iters = max_iters;
        for (int i = 0; i < 8; ++i) c->ph_ns[i] = 0;
        c->st_ext = c->st_bridge = c->st_root = c->st_ins = c->st_points = c->st_pairs = 0;
        c->st_nn_evals = c->st_nn_nodes = c->st_br_evals = c->st_br_nodes = 0;
        c->t_start = global_ns();
        c->t_first = 0;
        c->t_end = 0;
        R* x = fnode(S, 0);
        for (int j = 0; j < kDP; ++j) x[j] = R(0);
        for (int j = 0; j < kMaxDof; ++j) x[j] = S.qs[j];
        S.fpar[0] = -1;
        S.fcost[0] = R(0);
        S.fiter[0] = -1;
        S.bq_count[0] = S.bq_count[1] = 0;
        *S.path_len = 0;
    }
    for (int i = t; i <= S.N; i += blockDim.x) c->set_count[i] = 0;
    for (int i = t; i < S.N; i += blockDim.x) {
        c->n_s[i] = 0;
        c->snap_s[i] = 0;
        c->group_active[i] = 0;
        c->slot_has[i] = 0;
        c->slot_active[i] = 0;
        c->slot_T[i] = __longlong_as_double(0x7ff0000000000000LL);
        c->slot_k[i] = -1;
        c->slot_gen[i] = 0;
    }
    __syncthreads();
    if (t == 0) {
        if (S.variant == 0) {
            build_windows(S);
            partition(S, c->U);
            c->done = (c->Lg < fmin(c->H, c->U)) ? 0 : 1;
        } else {
            // Reading (root initialisation): the grid indices of [L_grid, H) are
            // split into N equal integer ranges; slot i takes the first
            // collision-free goal check of its range, scanning upward.
            long long K = c->kend - c->kmin;
            for (int i = 0; i < S.N; ++i) {
                long long a = c->kmin + (K * i) / S.N;
                long long b = c->kmin + (K * (i + 1)) / S.N;
                for (long long k = a; k < b; ++k) {
                    if (k - c->kmin < c->nk && S.gfree[k - c->kmin]) {
                        c->slot_has[i] = 1;
                        c->slot_active[i] = 1;
                        c->slot_k[i] = k;
                        c->slot_T[i] = grid_t<R>(k, c->dt);
                        c->slot_gen[i] = 0;
                        install_root(S, i, c->slot_T[i], 0, -1);
                        break;
                    }
                }
            }
            c->done = 0;
        }
        if (max_iters <= 0) c->done = 1;
    }
}

// ---------------------------------------------------------------------------
// Steering and edge entries. Worker w owns extension-batch entries 2w (the
// point check of its sampled goal root, interval root only) and 2w+1 (the
// extension edge); a count of 0 leaves an entry out of the batch.
// ---------------------------------------------------------------------------
// Check points of the edge (qa, ta) -> (qb, tb): ceil(L / res - 1e-3), at
// least 1, with L the larger of the configuration length and v_max |tb - ta|;
// working precision, rows held in registers.
template <typename R>
__device__ __forceinline__ int check_count_rows(const R (&qa)[kDP], R ta, const R (&qb)[kDP], R tb, int dof, R vmax,
                                                R res) {
    R s2 = R(0);
#pragma unroll
    for (int j = 0; j < kMaxDof; ++j) {
        if (j < dof) {
            R e = qb[j] - qa[j];
            s2 += e * e;
        }
    }
    R dt = tb - ta;
    R L = rsqrt_r(s2);
    R Lt = vmax * (dt < R(0) ? -dt : dt);
    if (Lt > L) L = Lt;
    R c = ceil(L / res - R(1e-3));
    return c < R(1) ? 1 : (int)c;
}

// Steer from x_n toward the worker's sample x_r (Algorithm 1 / Eq.
// max-speed-extension), check the horizon and emit the entries. Returns false
// when the attempt is skipped. Rows live in registers and move as vectors.
template <typename R>
__device__ __forceinline__ bool steer_and_emit(const Geom<R>& G, const State<R>& S, int w, int set, bool virt,
                                               const R (&xn)[kDP], const R (&xr)[kDP]) {
    const int dof = G.dof;
    R xw[kDP];
#pragma unroll
    for (int j = 0; j < kDP; ++j) xw[j] = R(0);
    R tnew;
    if (S.variant == 0) {
        const R tn = xn[kDP - 1], tr = xr[kDP - 1];
        const R D = qdist_rows(xn, xr, dof);
        if (virt) {
            // The virtual root is the sole source: rho must be finite.
            const R Delta = tn - tr;
            if (!(Delta > R(0)) || !(D <= G.vmax * Delta)) return false;
        }
        const R rho = rsqrt_r((D * D + G.vmax * G.vmax * (tr - tn) * (tr - tn)) / R(2));
        const R eta = (R)S.eta;
        const R alpha = (eta / rho) < R(1) ? (eta / rho) : R(1);
#pragma unroll
        for (int j = 0; j < kMaxDof; ++j)
            if (j < dof) xw[j] = xn[j] + alpha * (xr[j] - xn[j]);
        tnew = tn + alpha * (tr - tn);
    } else {
        const R D = qdist_rows(xn, xr, dof);
        if (!(D > R(0))) return false;
        const R eta = (R)S.eta;
        const R sc = (eta / D) < R(1) ? (eta / D) : R(1);
#pragma unroll
        for (int j = 0; j < kMaxDof; ++j)
            if (j < dof) xw[j] = xn[j] + sc * (xr[j] - xn[j]);
        const R Dn = qdist_rows(xn, xw, dof);
        tnew = xn[kDP - 1] + (set == 0 ? R(1) : R(-1)) * Dn / G.vmax;
    }
    xw[kDP - 1] = tnew;
    if (tnew < R(0) || tnew > (R)S.H) return false;
    st_row(S.w_xnew + (size_t)w * kDP, xw);
    st_row(S.w_xn + (size_t)w * kDP, xn);
    const R res = (R)S.res;
    if (S.variant == 0) {
        // Point check of the sampled goal root (q_g, T).
        const int e = 2 * w;
        R g[kDP];
#pragma unroll
        for (int j = 0; j < kDP; ++j) g[j] = R(0);
#pragma unroll
        for (int j = 0; j < kMaxDof; ++j) g[j] = S.qg[j];
        st_row(S.eqa + (size_t)e * kDP, g);
        st_row(S.eqb + (size_t)e * kDP, g);
        const R T = (R)S.w_T[w];
        S.eta_[e] = T;
        S.etb[e] = T;
        S.ecnt[e] = 1;
        S.w_root_edge[w] = e;
    }
    const int e = 2 * w + 1;
    st_row(S.eqa + (size_t)e * kDP, xn);
    st_row(S.eqb + (size_t)e * kDP, xw);
    S.eta_[e] = xn[kDP - 1];
    S.etb[e] = tnew;
    S.ecnt[e] = check_count_rows(xn, xn[kDP - 1], xw, tnew, dof, G.vmax, res);
    S.w_edge[w] = e;
    return true;
}

// ---------------------------------------------------------------------------
// k_sample: one thread per worker.
// ---------------------------------------------------------------------------
// One worker's sample (worker w of iteration k); act / nact: the active slots
// in slot order (recycling).
template <typename R>
__device__ __forceinline__ void sample_worker(const Geom<R>& G, const State<R>& S, int w, int k, const int* act,
                                              int nact) {
    const Ctl* c = S.ctl;
    const int dof = G.dof;
    const bool fwd = ((w + k) & 1) == 0;
    int status = kSkip, set = 0;
    R* xr = S.w_xr + (size_t)w * kDP;
    S.ecnt[2 * w] = 0;
    S.ecnt[2 * w + 1] = 0;
    S.ehit[2 * w] = 0;
    S.ehit[2 * w + 1] = 0;
    S.w_edge[w] = -1;
    S.w_root_edge[w] = -1;
    S.w_nnkey[w] = ~0ull;
    uint32_t d[20];
    philox4x32_10(0, (uint32_t)w, (uint32_t)k, S.problem_id, S.key0, S.key1, d);
    philox4x32_10(1, (uint32_t)w, (uint32_t)k, S.problem_id, S.key0, S.key1, d + 4);
    philox4x32_10(2, (uint32_t)w, (uint32_t)k, S.problem_id, S.key0, S.key1, d + 8);
    bool lrn = false;
    if (S.learned) {
        philox4x32_10(3, (uint32_t)w, (uint32_t)k, S.problem_id, S.key0, S.key1, d + 12);
        philox4x32_10(4, (uint32_t)w, (uint32_t)k, S.problem_id, S.key0, S.key1, d + 16);
        lrn = (d[12] >> 8) < kThrLearned;
    }
    R qr[kMaxDof];
#pragma unroll
    for (int j = 0; j < kMaxDof; ++j) qr[j] = (j < dof) ? G.qlo[j] + uni_r<R>(d[4 + j]) * (G.qhi[j] - G.qlo[j]) : R(0);
    if (lrn) learned_q(G, S, d, qr);
    R row[kDP];   // the sample x_r = (q_r, t_r) as stored
#pragma unroll
    for (int j = 0; j < kMaxDof; ++j) row[j] = qr[j];
    row[kDP - 1] = R(0);

    int tflags = (fwd ? kTrFwd : 0) | (lrn ? kTrLearned : 0), tgroup = -1, tcomp = -1;
    float tT = 0.f;
    if (S.variant == 0) {
        const int g = (int)(((unsigned long long)(d[0] >> 8) * (unsigned long long)S.N) >> 24);
        tgroup = g;
        bool guided;
        R Tr = sample_goal_time(S, g, d[1] >> 8, uni_r<R>(d[2]), guided);
        if (guided) tflags |= kTrGuided;
        if (lrn) {
            const R Tl = learned_T(S, d, tcomp);
            const R width = (R)c->width;
            const R glo = (R)c->Lg + (R)g * width;
            if (Tl >= glo && Tl < glo + width) {
                Tr = Tl;
                tflags |= kTrLearnedT;
            }
        }
        S.w_T[w] = Tr;
        tT = (float)Tr;
        // Conditional query time (Eq. conditional-query-time).
        const R lo = qdist_rows(S.qs, qr, dof) / G.vmax;
        const R hi = Tr - qdist_rows(qr, S.qg, dof) / G.vmax;
        if (!(lo > hi)) {
            // Slot 4 + d (selected without a dynamic index into d).
            uint32_t dword = d[4];
#pragma unroll
            for (int j = 1; j <= kMaxDof; ++j)
                if (j == dof) dword = d[4 + j];
            row[kDP - 1] = lo + uni_r<R>(dword) * (hi - lo);
            st_row(xr, row);
            tflags |= kTrSampled;
            set = fwd ? 0 : 1 + g;
            if (fwd) {
                status = kNN;
            } else {
                const bool use_new = (c->group_active[g] == 0) || ((d[3] >> 8) <= S.thr_new);
                status = use_new ? kVirtual : kNN;
            }
        }
    } else {
        int slot = -1;
        if (!fwd && nact > 0) slot = act[(w / 2) % nact];
        tgroup = slot;
        if (fwd || slot >= 0) {
            tflags |= kTrSampled;
            st_row(xr, row);
            set = fwd ? 0 : 1 + slot;
            status = kNN;
        }
    }
    if (status == kVirtual) {
        // The virtual root (q_g, T) is the sole source: steer at once.
        R xn[kDP];
#pragma unroll
        for (int j = 0; j < kMaxDof; ++j) xn[j] = S.qg[j];
        xn[kDP - 1] = (R)S.w_T[w];
        tflags |= kTrVirtual;
        if (!steer_and_emit(G, S, w, set, true, xn, row)) status = kSkip;
        else tflags |= kTrEmit;
    }
    if (int* tr = trace_rec(S, k, w)) {
        tr[kTfFlags] = tflags;
        tr[kTfGroup] = tgroup;
        tr[kTfParent] = -1;
        tr[kTfExtCount] = (tflags & kTrEmit) ? S.ecnt[2 * w + 1] : 0;
        tr[kTfBrSet] = -1;
        tr[kTfBrIdx] = -1;
        tr[kTfBrCount] = 0;
        tr[kTfInserted] = -1;
        tr[kTfComponent] = tcomp;
        tr[kTfGoalTime] = __float_as_int(tT);
    }
    S.w_status[w] = status;
    S.w_set[w] = set;
    S.w_parent[w] = -1;
    if (status == kNN) {
        int pos = atomicAdd(&S.ctl->set_count[set], 1);
        S.qlist[(size_t)set * S.W + pos] = w;
    }
}


// cta / ncta: this CTA's index among the CTAs sharing the step; workers are
// dealt in blocks of blockDim.x.
template <typename R>
__device__ __forceinline__ void sample_body(const Geom<R>& G, const State<R>& S, int cta, int ncta) {
    const Ctl* c = S.ctl;
    // Control words and the slot flags in one round of loads; nothing is
    // written before the termination flag is tested.
    const int done = c->done;
    const int k = c->iter;
    // Active-slot list (recycling) staged once per block.
    __shared__ int s_act[kMaxRoots];
    __shared__ int s_nact;
    if (S.variant != 0)
        for (int i = threadIdx.x; i < S.N; i += blockDim.x) s_act[i] = c->slot_active[i];
    if (done) return;
    if (S.variant != 0) {
        __syncthreads();
        if (threadIdx.x == 0) {
            int n = 0;
            for (int i = 0; i < S.N; ++i)
                if (s_act[i]) s_act[n++] = i;
            s_nact = n;
        }
        __syncthreads();
    }
    const int nact = S.variant != 0 ? s_nact : 0;
    for (int w = cta * blockDim.x + threadIdx.x; w < S.W; w += ncta * blockDim.x) sample_worker(G, S, w, k, s_act, nact);
    // The active-slot list is read until every worker of this block is done.
    __syncthreads();
}

// ---------------------------------------------------------------------------
// Tile scheduler shared by the NN and bridge scans.
// ---------------------------------------------------------------------------
// Node tiles in shared memory hold one row per node: DQ coordinates, time,
// and a flag/root-time word, padded to whole 16-byte vectors so that a scan
// step reads a node with 16-byte loads (two for DQ = 3 or 6, three for 7).
template <typename R, int DQ>
__host__ __device__ constexpr int tile_row() {
    return (int)((((DQ + 2) * sizeof(R) + 15) / 16) * 16 / sizeof(R));
}

template <typename R, int N>
__device__ __forceinline__ void lds_row(const R* row, R (&v)[N]) {
    static_assert((N * sizeof(R)) % 16 == 0, "tile rows are whole 16-byte vectors");
    if constexpr (sizeof(R) == 4) {
        const float4* p = reinterpret_cast<const float4*>(row);
#pragma unroll
        for (int k = 0; k < N / 4; ++k) {
            const float4 a = p[k];
            v[4 * k] = a.x;
            v[4 * k + 1] = a.y;
            v[4 * k + 2] = a.z;
            v[4 * k + 3] = a.w;
        }
    } else {
        const double2* p = reinterpret_cast<const double2*>(row);
#pragma unroll
        for (int k = 0; k < N / 2; ++k) {
            const double2 a = p[k];
            v[2 * k] = a.x;
            v[2 * k + 1] = a.y;
        }
    }
}

template <typename R, int N>
__device__ __forceinline__ void sts_row(R* row, const R (&v)[N]) {
    static_assert((N * sizeof(R)) % 16 == 0, "tile rows are whole 16-byte vectors");
    if constexpr (sizeof(R) == 4) {
#pragma unroll
        for (int k = 0; k < N / 4; ++k)
            reinterpret_cast<float4*>(row)[k] = make_float4(v[4 * k], v[4 * k + 1], v[4 * k + 2], v[4 * k + 3]);
    } else {
#pragma unroll
        for (int k = 0; k < N / 2; ++k) reinterpret_cast<double2*>(row)[k] = make_double2(v[2 * k], v[2 * k + 1]);
    }
}

// Tile row of a node: coordinates 0..DQ-1, time, flag word, zero padding.
template <typename R, int DQ, int N>
__device__ __forceinline__ void make_tile_row(const R* node, R flag, R (&v)[N]) {
    R x[kDP];
    ld_row(node, x);
#pragma unroll
    for (int j = 0; j < N; ++j) v[j] = R(0);
#pragma unroll
    for (int j = 0; j < DQ; ++j) v[j] = x[j];
    v[DQ] = x[kDP - 1];
    v[DQ + 1] = flag;
}

// Exclusive prefix of v[0..n) in place by the first warp of the block (lanes
// 0..31 call it together); returns the total to every calling lane.
__device__ __forceinline__ int warp_prefix_inplace(int* v, int n) {
    const int lane = threadIdx.x & 31;
    int carry = 0;
    for (int s0 = 0; s0 < n; s0 += 32) {
        const int s = s0 + lane;
        const int a = s < n ? v[s] : 0;
        int x = a;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (s < n) v[s] = carry + x - a;
        carry += __shfl_sync(0xffffffffu, x, 31);
    }
    return carry;
}

// Thread groups of kQT threads for the NN and bridge scans: the per-step
// kernels run one group per CTA (NG = 1); the persistent kernel runs two
// groups per 256-thread CTA (NG = 2), each a virtual CTA with its own shared
// tile and named barrier.
template <int NG>
__device__ __forceinline__ void group_sync() {
    if constexpr (NG == 1) {
        __syncthreads();
    } else {
        asm volatile("bar.sync %0, %1;" ::"r"(1 + (int)(threadIdx.x / kQT)), "n"(kQT) : "memory");
    }
}

struct TileSets {
    int pre[kMaxRoots + 2];  // tile prefix per set
    int nq[kMaxRoots + 1];
    int nn[kMaxRoots + 1];   // nodes
    int nt[kMaxRoots + 1];   // node tiles
    int nts[kMaxRoots + 1];  // nodes per tile
};

__device__ __forceinline__ void tiles_for(int nq, int n, int& nt, int& nts, int& tiles) {
    if (n <= 0 || nq <= 0) {
        nt = 0;
        nts = 0;
        tiles = 0;
        return;
    }
    nt = (n + kNodeTileMin - 1) / kNodeTileMin;
    if (nt > kMaxTiles) nt = kMaxTiles;
    nts = (n + nt - 1) / nt;
    nt = (n + nts - 1) / nts;
    tiles = ((nq + kQT - 1) / kQT) * nt;
}

// Lexicographic (k1, k2, idx) comparison.
template <typename R>
__device__ __forceinline__ bool key_less(R a1, R a2, int ai, R b1, R b2, int bi) {
    if (a1 != b1) return a1 < b1;
    if (a2 != b2) return a2 < b2;
    return ai < bi;
}

// Packed 64-bit NN key: non-negative FP32 key bits above the node index, so
// that an unsigned atomicMin keeps the smallest key and, among equal keys, the
// lowest index.
__device__ __forceinline__ unsigned long long pack_key(float k, int idx) {
    return ((unsigned long long)__float_as_uint(k) << 32) | (unsigned)idx;
}

// NN scan. Set 0 = forward arena; set 1+i = backward segment i. DQ = number of
// configuration coordinates compared (3 or 7; missing ones are zero).
// cta / ncta: this CTA's index among the CTAs sharing the step.
template <typename R, int DQ, int NG = 1>
__device__ __forceinline__ void nn_body(const Geom<R>& G, const State<R>& S, int cta, int ncta) {
    const Ctl* c = S.ctl;
    // Control words and the per-set counts in one round of loads; nothing is
    // written to global memory before the termination flag is tested.
    const int done = c->done;
    // U holds a value stored in the trees (or +inf), so it converts exactly.
    const R U0r = (R)c->U;
    __shared__ TileSets ts_[NG];
    constexpr int kRow = tile_row<R, DQ>();
    __shared__ __align__(16) R sx_[NG][kQT][kRow];
    __shared__ int s_last_[NG];
    const int grp = NG == 1 ? 0 : (int)threadIdx.x / kQT;
    TileSets& ts = ts_[grp];
    R (&sx)[kQT][kRow] = sx_[grp];
    int& s_last = s_last_[grp];
    const int t = NG == 1 ? (int)threadIdx.x : (int)threadIdx.x % kQT;
    const int vcta = cta * NG + grp, nvcta = ncta * NG;
    const int nsets = S.N + 1;
    const int titer = S.trace ? c->iter : -1;
    // One thread per set loads its counts, then the first warp forms the tile
    // prefix in shared memory.
    for (int s = t; s < nsets; s += kQT) {
        const int nq = c->set_count[s];
        const int n = s == 0 ? c->n_f : c->n_s[s - 1];
        int nt, nts, tiles;
        tiles_for(nq, n, nt, nts, tiles);
        ts.nq[s] = nq;
        ts.nn[s] = n;
        ts.nt[s] = nt;
        ts.nts[s] = nts;
        ts.pre[s] = tiles;
    }
    group_sync<NG>();
    if (done) return;
    if (t < 32) {
        const int acc = warp_prefix_inplace(ts.pre, nsets);
        if (t == 0) ts.pre[nsets] = acc;
    }
    group_sync<NG>();
    const int total = ts.pre[nsets];
    const R v2 = G.vmax * G.vmax;
    const bool interval = S.variant == 0;
    // The CTA scans its tiles chunk by chunk (kQT nodes each). The node rows
    // of the next chunk (of this tile, or the first of the CTA's next tile)
    // are loaded into registers while the current chunk is scanned, so only
    // the first chunk's global loads are exposed.
    auto tile_range = [&](int tl, int& s_, int& n0_, int& n1_) {
        s_ = 0;
        while (ts.pre[s_ + 1] <= tl) ++s_;
        const int ntile_ = (tl - ts.pre[s_]) % ts.nt[s_];
        n0_ = ntile_ * ts.nts[s_];
        n1_ = min(ts.nn[s_], n0_ + ts.nts[s_]);
    };
    R px[kDP];   // prefetched node row
    R ptro = R(0);  // and its root time (interval root, backward sets)
    auto prefetch = [&](int s_, int idx) {
        const R* b_ = s_ == 0 ? S.fx : S.bx + (size_t)(s_ - 1) * S.cap_s * kDP;
        ld_row(b_ + (size_t)idx * kDP, px);
        if (interval && s_ != 0) ptro = S.btroot[(size_t)(s_ - 1) * S.cap_s + idx];
    };
    if (vcta < total) {
        int s_, n0_, n1_;
        tile_range(vcta, s_, n0_, n1_);
        if (t < min(kQT, n1_ - n0_)) prefetch(s_, n0_ + t);
    }
    for (int tile = vcta; tile < total; tile += nvcta) {
        int s = 0;
        while (ts.pre[s + 1] <= tile) ++s;
        const int local = tile - ts.pre[s];
        const int nt = ts.nt[s];
        const int qt = local / nt, ntile = local % nt;
        const int qi = qt * kQT + t;
        const int w = qi < ts.nq[s] ? S.qlist[(size_t)s * S.W + qi] : -1;
        // The query row stays in registers for the scan and the steering.
        R xq[kDP];
#pragma unroll
        for (int j = 0; j < kDP; ++j) xq[j] = R(0);
        if (w >= 0) ld_row(S.w_xr + (size_t)w * kDP, xq);
        R q[DQ];
#pragma unroll
        for (int j = 0; j < DQ; ++j) q[j] = xq[j];
        const R tr = xq[kDP - 1];
        const int n0 = ntile * ts.nts[s];
        const int n1 = min(ts.nn[s], n0 + ts.nts[s]);
        const bool fwd = s == 0;
        R best = rinf<R>();
        int bidx = 0x7fffffff;
        for (int c0 = n0; c0 < n1; c0 += kQT) {
            const int cnt = min(kQT, n1 - c0);
            group_sync<NG>();
            if (t < cnt) {
                const bool active = !(interval && !fwd) || ptro < U0r;
                R v[kRow];
#pragma unroll
                for (int j = 0; j < kRow; ++j) v[j] = R(0);
#pragma unroll
                for (int j = 0; j < DQ; ++j) v[j] = px[j];
                v[DQ] = px[kDP - 1];
                v[DQ + 1] = active ? R(1) : R(0);
                sts_row(sx[t], v);
            }
            group_sync<NG>();
            {
                // Next chunk: the rest of this tile, else the CTA's next tile.
                int s_ = s, nc = c0 + kQT, ne = n1;
                bool more = nc < n1;
                if (!more && tile + nvcta < total) {
                    tile_range(tile + nvcta, s_, nc, ne);
                    more = true;
                }
                if (more && t < min(kQT, ne - nc)) prefetch(s_, nc + t);
            }
            if (w >= 0) {
                auto key_of = [&](int i) -> R {
                    R r[kRow];
                    lds_row<R, kRow>(sx[i], r);
                    R D2 = R(0);
#pragma unroll
                    for (int j = 0; j < DQ; ++j) {
                        R e = r[j] - q[j];
                        D2 += e * e;
                    }
                    if (!interval) return D2;
                    const R dt = tr - r[DQ];
                    const R Delta = fwd ? dt : -dt;
                    const bool ok = (r[DQ + 1] != R(0)) && (Delta > R(0)) && (D2 <= v2 * Delta * Delta);
                    return ok ? D2 + v2 * dt * dt : rinf<R>();
                };
                // Four independent key chains per step; updates in index order
                // keep the lowest index on ties.
                int i = 0;
                for (; i + 4 <= cnt; i += 4) {
                    const R k0 = key_of(i), k1 = key_of(i + 1), k2 = key_of(i + 2), k3 = key_of(i + 3);
                    if (k0 < best) { best = k0; bidx = c0 + i; }
                    if (k1 < best) { best = k1; bidx = c0 + i + 1; }
                    if (k2 < best) { best = k2; bidx = c0 + i + 2; }
                    if (k3 < best) { best = k3; bidx = c0 + i + 3; }
                }
                for (; i < cnt; ++i) {
                    const R k0 = key_of(i);
                    if (k0 < best) { best = k0; bidx = c0 + i; }
                }
            }
        }
        if constexpr (sizeof(R) == 4) {
            if (w >= 0 && best < rinf<R>()) atomicMin(S.w_nnkey + w, pack_key((float)best, bidx));
        } else {
            // FP64 keys do not fit one 64-bit word with the index: per-tile
            // partials, reduced in tile order by the last CTA of the query tile.
            if (w >= 0) {
                S.part_k2[(size_t)w * kMaxTiles + ntile] = best;
                S.part_idx[(size_t)w * kMaxTiles + ntile] = bidx;
            }
        }
        // The block's results are visible to thread 0 after the barrier; its
        // fence (cumulative) publishes them before the completion count.
        group_sync<NG>();
        if (t == 0) {
            const unsigned long long nq_t = (unsigned long long)min(kQT, ts.nq[s] - qt * kQT);
            atomicAdd(&S.ctl->st_nn_evals, nq_t * (unsigned long long)(n1 - n0));
            if (qt == 0) atomicAdd(&S.ctl->st_nn_nodes, (unsigned long long)(n1 - n0));
            __threadfence();
            int old = atomicAdd(&S.tile_cnt[s * kMaxQTiles + qt], 1);
            s_last = (old == nt - 1);
            if (s_last) __threadfence();
        }
        group_sync<NG>();
        if (s_last) {
            // Every tile of this query tile is done: decode the NN and steer.
            if (w >= 0) {
                int p;
                if constexpr (sizeof(R) == 4) {
                    const unsigned long long key = __ldcg(S.w_nnkey + w);
                    p = (key == ~0ull) ? -1 : (int)(unsigned)(key & 0xffffffffull);
                } else {
                    R b = rinf<R>();
                    int bi = 0x7fffffff;
                    for (int j = 0; j < nt; ++j) {
                        R kk = __ldcg(S.part_k2 + (size_t)w * kMaxTiles + j);
                        int ii = __ldcg(S.part_idx + (size_t)w * kMaxTiles + j);
                        if (kk < b || (kk == b && ii < bi)) {
                            b = kk;
                            bi = ii;
                        }
                    }
                    p = (b < rinf<R>()) ? bi : -1;
                }
                S.w_parent[w] = p;
                bool ok = p >= 0;
                if (ok) {
                    R xn[kDP];
                    ld_row(s == 0 ? fnode(S, p) : bnode(S, s - 1, p), xn);
                    ok = steer_and_emit(G, S, w, s, false, xn, xq);
                }
                if (!ok) S.w_status[w] = kSkip;
                if (int* tr = trace_rec(S, titer, w)) {
                    tr[kTfParent] = p;
                    if (ok) {
                        tr[kTfFlags] |= kTrEmit;
                        tr[kTfExtCount] = S.ecnt[2 * w + 1];
                    }
                }
            }
            if (t == 0) S.tile_cnt[s * kMaxQTiles + qt] = 0;
        }
    }
}

// ---------------------------------------------------------------------------
// Block-level helpers for the single-CTA kernels.
// ---------------------------------------------------------------------------
__device__ __forceinline__ long long cta_exclusive_scan(long long v, long long* sh, long long* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long x = v;
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        long long y = lane < nw ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            long long z = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += z;
        }
        if (lane < nw) sh[lane] = y;
    }
    __syncthreads();
    const long long before = (warp > 0 ? sh[warp - 1] : 0) + x - v;
    if (total) *total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before;
}

// ---------------------------------------------------------------------------
// k_insert: single CTA. Ordered insertion in worker order; also clears the
// per-worker bridge state of the iteration. Every load a chunk needs is issued
// in two rounds (the worker records with the control words, then the parents'
// records), and the bridge-query lists are filled in worker order from a scan.
// ---------------------------------------------------------------------------
// NT: threads of the (single) CTA that runs the step.
template <typename R, int NT = kCtaThreads>
__device__ __forceinline__ void insert_body(const Geom<R>& G, const State<R>& S) {
    Ctl* c = S.ctl;
    constexpr int kNW = NT / 32;
    static_assert(NT % 32 == 0 && kNW <= 32, "whole warps, at most 32");
    __shared__ int wt[kNW][kMaxRoots + 1];
    __shared__ int base[kMaxRoots + 1];
    __shared__ long long sh[32];
    __shared__ int tree_base;
    __shared__ int overflow;
    __shared__ long long bq_base;   // forward count (low 32 bits), backward count (high)
    __shared__ unsigned long long n_ins_total, n_ext_total;
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    const int nsets = S.N + 1;
    const int dof = G.dof;
    const int done = c->done;
    const int iter = c->iter;
    const int n_trees = c->n_trees;
    for (int s = t; s < nsets; s += blockDim.x) base[s] = s == 0 ? c->n_f : c->n_s[s - 1];
    if (t == 0) {
        tree_base = n_trees;
        overflow = 0;
        bq_base = 0;
        n_ins_total = 0;
        n_ext_total = 0;
    }
    for (int r0 = 0; r0 < S.W; r0 += NT) {
        const int w = r0 + t;
        // Round 1: the worker's records (entries of worker w sit at 2w, 2w+1).
        int e = -1, re = -1, h_root = 0, h_ext = 0, wset = -1, wst = 0, p = -1;
        R xw[kDP];
#pragma unroll
        for (int j = 0; j < kDP; ++j) xw[j] = R(0);
        if (w < S.W) {
            e = S.w_edge[w];
            re = S.w_root_edge[w];
            h_root = S.ehit[2 * w];
            h_ext = S.ehit[2 * w + 1];
            wset = S.w_set[w];
            wst = S.w_status[w];
            p = S.w_parent[w];
            ld_row(S.w_xnew + (size_t)w * kDP, xw);
        }
        if (r0 == 0) {
            __syncthreads();   // base[], tree_base and the counters are set
            if (done) return;
            for (int s = t; s < nsets; s += blockDim.x) {
                if (s == 0) c->snap_f = base[0];
                else c->snap_s[s - 1] = base[s];
            }
        }
        int ok = 0, nodes = 0, set = -1, virt = 0, ext = 0;
        if (w < S.W) {
            S.b_idx[w] = -1;
            S.w_bedge[w] = -1;
            S.bcnt[w] = 0;
            S.bhit[w] = 0;
            reinterpret_cast<ulonglong2*>(S.bkey)[w] = make_ulonglong2(~0ull, ~0ull);
            if (e >= 0) {
                const bool root_ok = re < 0 || h_root == 0;
                ext = root_ok ? 1 : 0;
                ok = root_ok && h_ext == 0;
            }
            if (ok) {
                set = wset;
                virt = wst == kVirtual;
                nodes = virt ? 2 : 1;
            }
        }
        // Round 2: the parent's record (or the virtual root's time), in flight
        // during the scans below.
        R pcost = R(0), ptroot = R(0), T = R(0);
        int ptree = 0;
        R px[kDP];
#pragma unroll
        for (int j = 0; j < kDP; ++j) px[j] = R(0);
        if (ok) {
            if (set == 0) {
                pcost = S.fcost[p];
                ld_row(fnode(S, p), px);
            } else if (virt) {
                T = S.w_T[w];
            } else {
                const size_t op = bofs(S, set - 1, p);
                pcost = S.bcost[op];
                ptroot = S.btroot[op];
                ptree = S.btree[op];
                ld_row(bnode(S, set - 1, p), px);
            }
        }
        // Rank among earlier lanes of this warp in the same set (weights 1 or 2).
        const unsigned same = __match_any_sync(0xffffffffu, set);
        const unsigned lt = (1u << lane) - 1u;
        const unsigned b0 = __ballot_sync(0xffffffffu, nodes & 1);
        const unsigned b1 = __ballot_sync(0xffffffffu, (nodes >> 1) & 1);
        const int in_warp = __popc(same & lt & b0) + 2 * __popc(same & lt & b1);
        const bool last_of_set = ((same >> lane) >> 1) == 0;  // highest lane of its group
        for (int s = t; s < kNW * nsets; s += NT) wt[s / nsets][s % nsets] = 0;
        __syncthreads();
        if (set >= 0 && last_of_set) wt[warp][set] = in_warp + nodes;
        __syncthreads();
        // Per set, exclusive scan over the warps' counts: one warp per set,
        // lane = warp index.
        for (int s = warp; s < nsets; s += kNW) {
            const int v = lane < kNW ? wt[lane][s] : 0;
            int x = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, x, o);
                if (lane >= o) x += y;
            }
            const int b = base[s];
            if (lane < kNW) wt[lane][s] = b + x - v;
            const int tot = __shfl_sync(0xffffffffu, x, 31);
            __syncwarp();
            if (lane == 0) base[s] = b + tot;
        }
        // Tree ids for materialised virtual roots, in worker order.
        long long tot_v;
        const long long vrank = cta_exclusive_scan(virt, sh, &tot_v);
        const int my_tree = tree_base + (int)vrank;
        int idx = ok ? wt[warp][set] + in_warp : 0;
        bool ins = false;
        if (ok) {
            if (set == 0) ins = idx + 1 <= S.cap_f;
            else ins = idx + nodes <= S.cap_s && !(virt && my_tree >= S.cap_trees);
        }
        // Bridge-query positions: forward insertions count in the low word,
        // backward ones in the high word.
        const long long flag = ins ? (set == 0 ? 1LL : (1LL << 32)) : 0LL;
        long long tot_q;
        const long long qrank = cta_exclusive_scan(flag, sh, &tot_q) + bq_base;
        __syncthreads();
        if (t == 0) {
            tree_base += (int)tot_v;
            bq_base += tot_q;
        }
        if (ok && !ins) overflow = 1;
        if (w < S.W) {
            if (int* tr = trace_rec(S, iter, w)) {
                int f = 0;
                if (re >= 0 && h_root) f |= kTrRootHit;
                if (e >= 0 && h_ext) f |= kTrExtHit;
                if (ins) f |= kTrInserted;
                tr[kTfFlags] |= f;
                tr[kTfInserted] = ins ? (set == 0 ? idx : idx + (virt ? 1 : 0)) : -1;
            }
        }
        if (ins) {
            if (set == 0) {
                st_row(fnode(S, idx), xw);
                S.fpar[idx] = p;
                S.fcost[idx] = pcost + qdist_rows(px, xw, dof);
                S.fiter[idx] = iter;
                S.w_ins[w] = idx;
                S.bq_list[S.W + (int)(qrank & 0xffffffffLL)] = w;
            } else {
                const int seg = set - 1;
                if (virt) {
                    // The new root (q_g, T) is the parent: its row stays in registers.
#pragma unroll
                    for (int j = 0; j < kDP; ++j) px[j] = R(0);
#pragma unroll
                    for (int j = 0; j < kMaxDof; ++j) px[j] = S.qg[j];
                    px[kDP - 1] = (R)T;
                    st_row(bnode(S, seg, idx), px);
                    size_t o = bofs(S, seg, idx);
                    S.bpar[o] = -1;
                    S.bcost[o] = R(0);
                    S.btroot[o] = (R)T;
                    S.btree[o] = my_tree;
                    S.biter[o] = iter;
                    S.tree_group[my_tree] = seg;
                    S.tree_T[my_tree] = (double)(R)T;  // as stored in the nodes
                    atomicAdd(&c->group_active[seg], 1);
                    pcost = R(0);
                    ptroot = (R)T;
                    ptree = my_tree;
                    p = idx;
                    ++idx;
                }
                st_row(bnode(S, seg, idx), xw);
                const size_t o = bofs(S, seg, idx);
                S.bpar[o] = p;
                S.bcost[o] = pcost + qdist_rows(px, xw, dof);
                S.btroot[o] = ptroot;
                S.btree[o] = ptree;
                S.biter[o] = iter;
                S.w_ins[w] = idx;
                S.bq_list[(int)(qrank >> 32)] = w;
            }
        } else if (w < S.W) {
            S.w_ins[w] = -1;
        }
        // statistics
        const unsigned bo = __ballot_sync(0xffffffffu, ok);
        const unsigned be = __ballot_sync(0xffffffffu, ext);
        if (lane == 0) {
            atomicAdd(&n_ins_total, (unsigned long long)__popc(bo));
            atomicAdd(&n_ext_total, (unsigned long long)__popc(be));
        }
        __syncthreads();
    }
    __syncthreads();
    for (int s = t; s < nsets; s += blockDim.x) {
        if (s == 0) c->n_f = min(base[0], S.cap_f);
        else c->n_s[s - 1] = min(base[s], S.cap_s);
    }
    if (t == 0) {
        c->n_trees = min(tree_base, S.cap_trees);
        c->st_ins += n_ins_total;
        c->st_ext += n_ext_total;
        S.bq_count[0] = (int)(bq_base >> 32);
        S.bq_count[1] = (int)(bq_base & 0xffffffffLL);
        if (overflow) {
            c->err |= kErrCapacity;
            c->done = 1;
        }
    }
}

// Candidate (U, C) of worker w's bridge and, if it improves the incumbent at
// the start of the iteration, its edge entry (entry index w of the bridge batch).
template <typename R>
__device__ __forceinline__ int bridge_emit(const Geom<R>& G, const State<R>& S, int w, R U0, R C0) {
    const bool fwd = S.w_set[w] == 0;
    const R* f;
    const R* b;
    R cf, cb, troot;
    if (fwd) {
        f = fnode(S, S.w_ins[w]);
        cf = S.fcost[S.w_ins[w]];
        const size_t o = bofs(S, S.b_set[w], S.b_idx[w]);
        b = bnode(S, S.b_set[w], S.b_idx[w]);
        cb = S.bcost[o];
        troot = S.btroot[o];
    } else {
        const int seg = S.w_set[w] - 1;
        const size_t o = bofs(S, seg, S.w_ins[w]);
        b = bnode(S, seg, S.w_ins[w]);
        cb = S.bcost[o];
        troot = S.btroot[o];
        f = fnode(S, S.b_idx[w]);
        cf = S.fcost[S.b_idx[w]];
    }
    R fr[kDP], br[kDP];
    ld_row(f, fr);
    ld_row(b, br);
    const R D = qdist_rows(fr, br, G.dof);
    const R Uc = troot;
    const R Cc = (cf + D) + cb;
    const bool improves = (Uc < U0) || (Uc == U0 && Cc < C0);
    if (!improves) return 0;
    S.b_U[w] = Uc;
    S.b_C[w] = Cc;
    st_row(S.bqa + (size_t)w * kDP, fr);
    st_row(S.bqb + (size_t)w * kDP, br);
    S.bta[w] = fr[kDP - 1];
    S.btb[w] = br[kDP - 1];
    S.bcnt[w] = check_count_rows(fr, fr[kDP - 1], br, br[kDP - 1], G.dof, G.vmax, (R)S.res);
    S.w_bedge[w] = w;
    return 1;
}

// Minimum of a 128-bit key (high word first) by compare-and-swap. Keys only
// decrease, so a failed exchange means another writer stored a smaller key:
// the loop ends after at most one retry per competing writer (the bound only
// guards against a corrupted key). The first exchange assumes the reset value,
// so no non-atomic read of the key is trusted.
__device__ __forceinline__ bool cas_min_u128(unsigned long long* base, int w, unsigned long long hi,
                                             unsigned long long lo) {
    unsigned __int128* a = reinterpret_cast<unsigned __int128*>(base) + w;
    const unsigned __int128 v = ((unsigned __int128)hi << 64) | lo;
    unsigned __int128 cur = ~(unsigned __int128)0;
    for (int it = 0; it < (1 << 16); ++it) {
        if (!(v < cur)) return true;
        const unsigned __int128 prev = atomicCAS(a, cur, v);
        if (prev == cur) return true;
        cur = prev;
    }
    return false;
}

// ---------------------------------------------------------------------------
// k_bridge: best-ranked admissible vertex of the opposite start-of-iteration set.
// Set 0: queries = backward-inserted nodes, vertices = forward arena [0, snap_f).
// Set 1: queries = forward-inserted nodes, vertices = all backward segments
//        [0, snap_s[i]) concatenated in segment order; active iff troot < U.
// Rank: (arrival time, rho^2, index) lexicographic. FP32 tiles merge their
// best into one 128-bit key per query (compare-and-swap minimum); FP64 tiles
// leave partials that the last CTA of the query tile reduces in tile order.
// The last CTA of a query tile emits the bridge edges.
// ---------------------------------------------------------------------------
template <typename R, int DQ, int NG = 1>
__device__ __forceinline__ void bridge_body(const Geom<R>& G, const State<R>& S, int cta, int ncta) {
    Ctl* c = S.ctl;
    // Control words, segment sizes and query counts in one round of loads;
    // nothing is written to global memory before the termination flag is tested.
    const int done = c->done;
    const R U0r = (R)c->U, C0r = (R)c->C;
    struct BridgeSh {
        int seg_pre[kMaxRoots + 1];
        int s_nq[2], s_nn[2], s_nt[2], s_nts[2], s_pre[3];
        int s_last, s_emitted;
    };
    __shared__ BridgeSh bsh_[NG];
    constexpr int kRow = tile_row<R, DQ>();
    __shared__ __align__(16) R sx_[NG][kQT][kRow];
    const int grp = NG == 1 ? 0 : (int)threadIdx.x / kQT;
    BridgeSh& bsh = bsh_[grp];
    int (&seg_pre)[kMaxRoots + 1] = bsh.seg_pre;
    int (&s_nq)[2] = bsh.s_nq;
    int (&s_nn)[2] = bsh.s_nn;
    int (&s_nt)[2] = bsh.s_nt;
    int (&s_nts)[2] = bsh.s_nts;
    int (&s_pre)[3] = bsh.s_pre;
    int& s_last = bsh.s_last;
    int& s_emitted = bsh.s_emitted;
    R (&sx)[kQT][kRow] = sx_[grp];
    const int t = NG == 1 ? (int)threadIdx.x : (int)threadIdx.x % kQT;
    const int vcta = cta * NG + grp, nvcta = ncta * NG;
    const int titer = S.trace ? c->iter : -1;
    for (int i = t; i < S.N; i += kQT) seg_pre[i] = c->snap_s[i];
    int nq0 = 0, nq1 = 0, nf = 0;
    if (t == 0) {
        nq0 = S.bq_count[0];
        nq1 = S.bq_count[1];
        nf = c->snap_f;
    }
    group_sync<NG>();
    if (done) return;
    if (t < 32) {
        const int acc = warp_prefix_inplace(seg_pre, S.N);
        if (t == 0) seg_pre[S.N] = acc;
    }
    if (t == 0) {
        const int acc = seg_pre[S.N];
        int tacc = 0;
        for (int s = 0; s < 2; ++s) {
            int nq = s == 0 ? nq0 : nq1;
            int n = s == 0 ? nf : acc;
            int nt, nts, tiles;
            tiles_for(nq, n, nt, nts, tiles);
            s_nq[s] = nq;
            s_nn[s] = n;
            s_nt[s] = nt;
            s_nts[s] = nts;
            s_pre[s] = tacc;
            tacc += tiles;
        }
        s_pre[2] = tacc;
        s_emitted = 0;
    }
    group_sync<NG>();
    const int total = s_pre[2];
    const R v2 = G.vmax * G.vmax;
    // Chunks of kQT nodes as in the NN scan: the next chunk's node rows (and
    // root times) are loaded into registers while the current one is ranked.
    auto tile_range = [&](int tl, int& s_, int& n0_, int& n1_) {
        s_ = tl < s_pre[1] ? 0 : 1;
        const int ntile_ = (tl - s_pre[s_]) % s_nt[s_];
        n0_ = ntile_ * s_nts[s_];
        n1_ = min(s_nn[s_], n0_ + s_nts[s_]);
    };
    R px[kDP];      // prefetched node row
    R ptro = R(0);  // its root time (0 for forward nodes)
    auto prefetch = [&](int s_, int li) {
        if (s_ == 0) {
            ld_row(fnode(S, li), px);
            ptro = R(0);
        } else {
            int sg = 0;
            while (seg_pre[sg + 1] <= li) ++sg;
            const int i = li - seg_pre[sg];
            ld_row(bnode(S, sg, i), px);
            ptro = S.btroot[bofs(S, sg, i)];
        }
    };
    if (vcta < total) {
        int s_, n0_, n1_;
        tile_range(vcta, s_, n0_, n1_);
        if (t < min(kQT, n1_ - n0_)) prefetch(s_, n0_ + t);
    }
    for (int tile = vcta; tile < total; tile += nvcta) {
        const int s = tile < s_pre[1] ? 0 : 1;
        const int local = tile - s_pre[s];
        const int nt = s_nt[s];
        const int qt = local / nt, ntile = local % nt;
        const int qi = qt * kQT + t;
        const int w = qi < s_nq[s] ? S.bq_list[(size_t)s * S.W + qi] : -1;
        R xq[kDP];
#pragma unroll
        for (int j = 0; j < kDP; ++j) xq[j] = R(0);
        if (w >= 0) ld_row(S.w_xnew + (size_t)w * kDP, xq);
        R q[DQ];
#pragma unroll
        for (int j = 0; j < DQ; ++j) q[j] = xq[j];
        const R tq = xq[kDP - 1];
        const int n0 = ntile * s_nts[s];
        const int n1 = min(s_nn[s], n0 + s_nts[s]);
        R b1 = rinf<R>(), b2 = rinf<R>();
        int bidx = 0x7fffffff;
        for (int c0 = n0; c0 < n1; c0 += kQT) {
            const int cnt = min(kQT, n1 - c0);
            group_sync<NG>();
            if (t < cnt) {
                const bool active = s == 0 || ptro < U0r;
                R v[kRow];
#pragma unroll
                for (int j = 0; j < kRow; ++j) v[j] = R(0);
#pragma unroll
                for (int j = 0; j < DQ; ++j) v[j] = px[j];
                v[DQ] = px[kDP - 1];
                v[DQ + 1] = active ? ptro : rinf<R>();
                sts_row(sx[t], v);
            }
            group_sync<NG>();
            {
                // Next chunk: the rest of this tile, else the CTA's next tile.
                int s_ = s, nc = c0 + kQT, ne = n1;
                bool more = nc < n1;
                if (!more && tile + nvcta < total) {
                    tile_range(tile + nvcta, s_, nc, ne);
                    more = true;
                }
                if (more && t < min(kQT, ne - nc)) prefetch(s_, nc + t);
            }
            if (w >= 0) {
                // Rank key of vertex i: (arrival time, rho^2); rho^2 = inf when
                // the vertex is inactive or not admissible.
                auto key_of = [&](int i, R& k1) -> R {
                    R r[kRow];
                    lds_row<R, kRow>(sx[i], r);
                    const R tro = r[DQ + 1];
                    k1 = s == 0 ? R(0) : tro;
                    R D2 = R(0);
#pragma unroll
                    for (int j = 0; j < DQ; ++j) {
                        R e = r[j] - q[j];
                        D2 += e * e;
                    }
                    // s = 0: vertex earlier than the query; s = 1: later.
                    const R dt = s == 0 ? tq - r[DQ] : r[DQ] - tq;
                    const bool ok = (tro < rinf<R>()) && (dt > R(0)) && (D2 <= v2 * dt * dt);
                    return ok ? D2 + v2 * dt * dt : rinf<R>();
                };
                auto take = [&](R k1, R k2, int idx) {
                    if (k2 < rinf<R>() && key_less(k1, k2, idx, b1, b2, bidx)) {
                        b1 = k1;
                        b2 = k2;
                        bidx = idx;
                    }
                };
                int i = 0;
                for (; i + 4 <= cnt; i += 4) {
                    R a1, b1_, c1, d1;
                    const R a2 = key_of(i, a1), b2_ = key_of(i + 1, b1_), c2 = key_of(i + 2, c1),
                            d2 = key_of(i + 3, d1);
                    take(a1, a2, c0 + i);
                    take(b1_, b2_, c0 + i + 1);
                    take(c1, c2, c0 + i + 2);
                    take(d1, d2, c0 + i + 3);
                }
                for (; i < cnt; ++i) {
                    R a1;
                    const R a2 = key_of(i, a1);
                    take(a1, a2, c0 + i);
                }
            }
        }
        if constexpr (sizeof(R) == 4) {
            // FP32: (k1, k2, index) fits 128 bits; non-negative floats order
            // like their bit patterns (+ 0 turns a -0 into +0).
            if (w >= 0 && b2 < rinf<R>()) {
                const unsigned long long hi = ((unsigned long long)__float_as_uint((float)b1 + 0.0f) << 32) |
                                              (unsigned long long)__float_as_uint((float)b2 + 0.0f);
                if (!cas_min_u128(S.bkey, w, hi, (unsigned long long)(unsigned)bidx)) atomicOr(&c->err, kErrInternal);
            }
        } else {
            // FP64 keys do not fit: per-tile partials, reduced in tile order
            // by the last CTA of the query tile.
            if (w >= 0) {
                S.part_k1[(size_t)w * kMaxTiles + ntile] = b1;
                S.part_k2[(size_t)w * kMaxTiles + ntile] = b2;
                S.part_idx[(size_t)w * kMaxTiles + ntile] = bidx;
            }
        }
        group_sync<NG>();
        if (t == 0) {
            const unsigned long long nq_t = (unsigned long long)min(kQT, s_nq[s] - qt * kQT);
            atomicAdd(&c->st_br_evals, nq_t * (unsigned long long)(n1 - n0));
            if (qt == 0) atomicAdd(&c->st_br_nodes, (unsigned long long)(n1 - n0));
            __threadfence();
            int old = atomicAdd(&S.btile_cnt[s * kMaxQTiles + qt], 1);
            s_last = (old == nt - 1);
            if (s_last) __threadfence();
        }
        group_sync<NG>();
        if (s_last) {
            int emitted = 0;
            if (w >= 0) {
                R k1 = rinf<R>(), k2 = rinf<R>();
                int bi = 0x7fffffff;
                if constexpr (sizeof(R) == 4) {
                    const ulonglong2 kv = __ldcg(reinterpret_cast<const ulonglong2*>(S.bkey) + w);
                    if (kv.x != ~0ull || kv.y != ~0ull) {
                        k1 = __uint_as_float((unsigned)(kv.y >> 32));
                        k2 = __uint_as_float((unsigned)(kv.y & 0xffffffffull));
                        bi = (int)(unsigned)kv.x;
                    }
                } else {
                    const R* p1 = S.part_k1 + (size_t)w * kMaxTiles;
                    const R* p2 = S.part_k2 + (size_t)w * kMaxTiles;
                    const int* pi = S.part_idx + (size_t)w * kMaxTiles;
                    // Groups of 8 independent loads per round trip, in tile order.
                    for (int j0 = 0; j0 < nt; j0 += 8) {
                        R a1[8], a2[8];
                        int ai[8];
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const int j = j0 + u < nt ? j0 + u : nt - 1;
                            a1[u] = __ldcg(p1 + j);
                            a2[u] = __ldcg(p2 + j);
                            ai[u] = __ldcg(pi + j);
                        }
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            if (j0 + u < nt && key_less(a1[u], a2[u], ai[u], k1, k2, bi)) {
                                k1 = a1[u];
                                k2 = a2[u];
                                bi = ai[u];
                            }
                        }
                    }
                }
                if (k2 < rinf<R>()) {
                    if (s == 0) {
                        S.b_set[w] = -1;
                        S.b_idx[w] = bi;
                    } else {
                        int sg = 0;
                        while (seg_pre[sg + 1] <= bi) ++sg;
                        S.b_set[w] = sg;
                        S.b_idx[w] = bi - seg_pre[sg];
                    }
                    emitted = bridge_emit(G, S, w, U0r, C0r);
                    if (int* tr = trace_rec(S, titer, w)) {
                        tr[kTfFlags] |= kTrBrCand | (emitted ? kTrBrEmit : 0);
                        tr[kTfBrSet] = S.b_set[w];
                        tr[kTfBrIdx] = S.b_idx[w];
                        if (emitted) tr[kTfBrCount] = S.bcnt[w];
                    }
                }
            }
            if (emitted) atomicAdd(&s_emitted, 1);
            if (t == 0) S.btile_cnt[s * kMaxQTiles + qt] = 0;
        }
    }
    group_sync<NG>();
    if (t == 0 && s_emitted) atomicAdd(&c->st_bridge, (unsigned long long)s_emitted);
}

// ---------------------------------------------------------------------------
// k_publish: single CTA. Lexicographic min of (U, C, worker); incumbent;
// allocation update.
// ---------------------------------------------------------------------------
template <typename R>
__device__ __forceinline__ void publish_body(const Geom<R>& G, const State<R>& S) {
    Ctl* c = S.ctl;
    // The termination flag is read with the candidates (one round of loads);
    // nothing is written before it is tested.
    const int done = c->done;
    __shared__ R rU[kCtaThreads / 32], rC[kCtaThreads / 32];
    __shared__ int rW[kCtaThreads / 32];
    __shared__ int rRec[kCtaThreads / 32][4];
    __shared__ int s_counts[kMaxRoots];
    __shared__ double sU, sC;
    __shared__ int s_iter, s_first, s_err, s_decreased;
    __shared__ int s_donors[kMaxRoots];
    __shared__ long long s_held[kMaxRoots];
    const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
    // Control fields staged in parallel with the candidate loads.
    if (t == 0) sU = c->U;
    if (t == 32) sC = c->C;
    if (t == 64) s_iter = c->iter;
    if (t == 96) s_first = c->first_iter;
    if (t == 128) s_err = c->err;
    // Each lane keeps its best candidate with the records the incumbent update
    // needs, so the winner needs no further load.
    R bU = rinf<R>(), bC = rinf<R>();
    int bw = 0x7fffffff, bws = 0, bwi = -1, bbs = -1, bbi = -1;
    const int titer = (S.trace && !done) ? c->iter : -1;
    for (int w = t; w < S.W; w += blockDim.x) {
        // Bridge entry of worker w is entry w; all loads independent.
        const int e = S.w_bedge[w];
        const int h = S.bhit[w];
        const R U = S.b_U[w], C = S.b_C[w];
        const int ws = S.w_set[w], wi = S.w_ins[w], bs = S.b_set[w], bi = S.b_idx[w];
        if (e >= 0 && h)
            if (int* tr = trace_rec(S, titer, w)) tr[kTfFlags] |= kTrBrHit;
        if (e < 0 || h) continue;
        if (U < bU || (U == bU && (C < bC || (C == bC && w < bw)))) {
            bU = U;
            bC = C;
            bw = w;
            bws = ws;
            bwi = wi;
            bbs = bs;
            bbi = bi;
        }
    }
    auto reduce_warp = [&]() {
        for (int o = 16; o > 0; o >>= 1) {
            const R U = __shfl_xor_sync(0xffffffffu, bU, o);
            const R C = __shfl_xor_sync(0xffffffffu, bC, o);
            const int ww = __shfl_xor_sync(0xffffffffu, bw, o);
            const int ws = __shfl_xor_sync(0xffffffffu, bws, o), wi = __shfl_xor_sync(0xffffffffu, bwi, o);
            const int bs = __shfl_xor_sync(0xffffffffu, bbs, o), bi = __shfl_xor_sync(0xffffffffu, bbi, o);
            if (U < bU || (U == bU && (C < bC || (C == bC && ww < bw)))) {
                bU = U;
                bC = C;
                bw = ww;
                bws = ws;
                bwi = wi;
                bbs = bs;
                bbi = bi;
            }
        }
    };
    reduce_warp();
    if (done) return;
    if (lane == 0) {
        rU[warp] = bU;
        rC[warp] = bC;
        rW[warp] = bw;
        rRec[warp][0] = bws;
        rRec[warp][1] = bwi;
        rRec[warp][2] = bbs;
        rRec[warp][3] = bbi;
    }
    __syncthreads();
    if (warp == 0) {
        const int nw = (int)(blockDim.x >> 5);
        bU = lane < nw ? rU[lane] : rinf<R>();
        bC = lane < nw ? rC[lane] : rinf<R>();
        bw = lane < nw ? rW[lane] : 0x7fffffff;
        bws = lane < nw ? rRec[lane][0] : 0;
        bwi = lane < nw ? rRec[lane][1] : -1;
        bbs = lane < nw ? rRec[lane][2] : -1;
        bbi = lane < nw ? rRec[lane][3] : -1;
        reduce_warp();
    }
    if (t == 0) {
        s_decreased = 0;
        if (bw != 0x7fffffff) {
            if (int* tr = trace_rec(S, s_iter, bw)) tr[kTfFlags] |= kTrWinner;
            s_decreased = bU < (R)sU;
            sU = (double)bU;
            sC = (double)bC;
            c->U = sU;
            c->C = sC;
            if (bws == 0) {
                c->inc_f = bwi;
                c->inc_s = bbs;
                c->inc_b = bbi;
            } else {
                c->inc_f = bbi;
                c->inc_s = bws - 1;
                c->inc_b = bwi;
            }
            if (s_first < 0) {
                c->first_iter = s_iter;
                c->t_first = global_ns();
            }
        }
    }
    __syncthreads();
    if (s_decreased) {
        if (S.variant == 0) {
            // Repartition; trees rooted at T >= U become inactive.
            for (int i = t; i < S.N; i += blockDim.x) s_counts[i] = 0;
            __syncthreads();
            const int ntr = c->n_trees;
            for (int i = t; i < ntr; i += blockDim.x)
                if (S.tree_T[i] < sU) atomicAdd(&s_counts[S.tree_group[i]], 1);
            __syncthreads();
            for (int i = t; i < S.N; i += blockDim.x) c->group_active[i] = s_counts[i];
            if (t == 0) partition(S, sU);
        } else if (t == 0) {
            if (S.variant == 1) {
                recycle(S, sU, s_donors, s_held);
            } else {
                // No recycling (the allocation ablation): the fixed forest only
                // loses the roots that can no longer improve U.
                Ctl* cc = S.ctl;
                for (int i = 0; i < S.N; ++i)
                    if (cc->slot_has[i] && cc->slot_T[i] >= sU) cc->slot_active[i] = 0;
            }
        }
    }
    __syncthreads();
    if (t == 0) {
        S.U_hist[s_iter] = sU;
        c->iter = s_iter + 1;
        S.bq_count[0] = S.bq_count[1] = 0;
        if (S.variant == 0) c->st_root += (unsigned long long)S.W;
        bool stop = s_iter + 1 >= c->max_iters || s_err != 0;
        if (c->budget_ns && global_ns() - c->t_start >= c->budget_ns) stop = true;
        if (S.variant == 0 && !(c->Lg < fmin(c->H, sU))) stop = true;
        if (stop) {
            c->done = 1;
            c->t_end = global_ns();
        }
    }
    for (int i = t; i <= S.N; i += blockDim.x) c->set_count[i] = 0;
}

// Path: forward chain from the start root to inc_f, then backward chain from
// inc_b to its root. One thread.
template <typename R>
__device__ __forceinline__ void extract_path_body(const State<R>& S) {
    // The forward branch (incumbent's forward node back to the start) and the
    // backward branch (its backward node up to the goal root) are walked once
    // each, concurrently, by the first lanes of two warps into shared index
    // lists; then every thread copies rows. Walks are bounded by the path
    // capacity (parents always precede children, so a longer walk cannot occur
    // in a consistent tree); a branch longer than the lists falls back to a
    // second walk by one thread.
    constexpr int kList = 512;
    __shared__ int s_idx[2][kList];
    __shared__ int s_len[2];
    const Ctl* c = S.ctl;
    const int t = threadIdx.x;
    const int inc_f = c->inc_f, inc_b = c->inc_b, inc_s = c->inc_s;
    if (inc_f < 0) {
        if (t == 0) *S.path_len = 0;
        return;
    }
    const int walker = blockDim.x >= 64 ? 32 : 0;  // thread of the backward walk
    if (t == 0) {
        int len = 0;
        for (int i = inc_f; i >= 0 && len <= S.path_cap; i = S.fpar[i]) {
            if (len < kList) s_idx[0][len] = i;
            ++len;
        }
        s_len[0] = len;
    }
    if (t == walker) {
        int len = 0;
        for (int i = inc_b; i >= 0 && len <= S.path_cap; i = S.bpar[bofs(S, inc_s, i)]) {
            if (len < kList) s_idx[1][len] = i;
            ++len;
        }
        s_len[1] = len;
    }
    __syncthreads();
    const int len_f = s_len[0], len_b = s_len[1];
    if (len_f + len_b > S.path_cap) {
        if (t == 0) *S.path_len = -(len_f + len_b);
        return;
    }
    if (len_f <= kList && len_b <= kList) {
        for (int k = t; k < len_f + len_b; k += blockDim.x) {
            const R* x = k < len_f ? fnode(S, s_idx[0][len_f - 1 - k]) : bnode(S, inc_s, s_idx[1][k - len_f]);
            for (int j = 0; j < kDP; ++j) S.path[(size_t)k * kDP + j] = x[j];
        }
    } else if (t == 0) {
        int k = len_f - 1;
        for (int i = inc_f; i >= 0; i = S.fpar[i], --k)
            for (int j = 0; j < kDP; ++j) S.path[(size_t)k * kDP + j] = fnode(S, i)[j];
        k = len_f;
        for (int i = inc_b; i >= 0; i = S.bpar[bofs(S, inc_s, i)], ++k)
            for (int j = 0; j < kDP; ++j) S.path[(size_t)k * kDP + j] = bnode(S, inc_s, i)[j];
    }
    if (t == 0) *S.path_len = len_f + len_b;
}

}  // namespace stp
