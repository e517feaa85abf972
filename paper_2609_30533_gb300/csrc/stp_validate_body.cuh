// Edge validation device code (collision checking of space-time edges
// against moving obstacles; Sec. "Simulation Protocol": every check point
// takes the obstacles where their trajectories put them at its own absolute
// time), shared by the stand-alone
// collision kernels and the persistent planner kernel.
//
// Mapping: a persistent grid walks the flat list of check points of a batch
// of edges, one check point per lane. Small batches (the planner's, offsets
// scanned into shared memory by every CTA) spread the whole flat range over
// all warps; large batches (precomputed offsets) go window by window, 256 edges
// per CTA window, with the window's offsets staged in shared memory. Either
// way a lane finds its edge by binary search in shared memory. A
// lane evaluates one check point completely: interpolate the edge in (q, t),
// run forward kinematics once, and test every robot sphere against every
// obstacle sphere. Obstacle positions at the lane's time are held in
// registers in chunks of MO obstacles; FK is amortised over all pairs.
// Robot spheres and obstacle trajectories are staged into shared memory by a
// single TMA bulk copy per CTA. FP32 CUDA-core arithmetic (no tensor cores:
// the pair tests are not a contraction).
//
// Algorithmic work per check point: S*M pair tests (8 flops each: 3 sub,
// 1 mul, 2 fma) + S sphere transforms + FK (d joint steps) + M interpolations.
//
// Verdict-only pair test. With positions taken relative to a reference point
// (the arm base, or the centre of a point robot's box), a robot sphere (c, r_s)
// and an obstacle (o, r_o) collide iff |c - o|^2 - (r_s + r_o)^2 < 0, i.e.
//   B_o + (-2 o).c + (-2 r_o) r_s  <  r_s^2 - |c|^2,   B_o = |o|^2 - r_o^2,
// which is four FMAs per pair against per-obstacle terms computed once per
// check point, plus one min per pair. In FP32 two pairs share each packed FMA
// (fma.rn.f32x2) and one three-input min; when all obstacles have one radius
// the r_s r_o term joins the per-sphere threshold and a pair costs three FMAs.
// Positions are O(1 m) relative to the reference, so the FP32 cancellation
// error near contact is about 1e-6 m; the clearance variant keeps the direct
// form |c - o| - r_s - r_o.
#pragma once

#include "stp_internal.cuh"

namespace stp {

// Per-check-point obstacle terms for the expanded pair test.
template <typename R, int MO>
struct ObsTerms {
    R ox[MO], oy[MO], oz[MO], ro[MO], B[MO];
};

template <typename R>
__device__ __forceinline__ R rmin(R a, R b) { return a < b ? a : b; }

// Packed FP32x2 helpers (Blackwell fma.rn.f32x2: two FP32 FMAs per
// instruction, each rounded once like the scalar FMA).
__device__ __forceinline__ unsigned long long pk2(float lo, float hi) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk2(unsigned long long v, float& lo, float& hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long ffma2(unsigned long long a, unsigned long long b,
                                                    unsigned long long c) {
    unsigned long long d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}

template <typename R, int MO>
__device__ __forceinline__ bool sphere_hits(R cx, R cy, R cz, R rs, const ObsTerms<R, MO>& O) {
    const R negA = rs * rs - (cx * cx + cy * cy + cz * cz);
    R m0 = rinf<R>(), m1 = rinf<R>();
#pragma unroll
    for (int j = 0; j < MO; j += 2) {
        R a = O.B[j];
        a = cx * O.ox[j] + a;
        a = cy * O.oy[j] + a;
        a = cz * O.oz[j] + a;
        a = rs * O.ro[j] + a;
        m0 = rmin(m0, a);
        if (j + 1 < MO) {
            R b = O.B[j + 1];
            b = cx * O.ox[j + 1] + b;
            b = cy * O.oy[j + 1] + b;
            b = cz * O.oz[j + 1] + b;
            b = rs * O.ro[j + 1] + b;
            m1 = rmin(m1, b);
        }
    }
    return rmin(m0, m1) < negA;
}

template <typename R, int MO, bool CLEAR>
__device__ __forceinline__ void test_sphere(R cx, R cy, R cz, R rs, const R (&ox)[MO], const R (&oy)[MO],
                                            const R (&oz)[MO], const R (&orr)[MO], bool& hit, R& clr) {
#pragma unroll
    for (int j = 0; j < MO; ++j) {
        R dx = cx - ox[j];
        R dy = cy - oy[j];
        R dz = cz - oz[j];
        R d2 = dx * dx + dy * dy + dz * dz;
        R rr = rs + orr[j];
        if (CLEAR) {
            R cl = rsqrt_r(d2) - rr;
            clr = cl < clr ? cl : clr;
        }
        hit = hit || (d2 < rr * rr);
    }
}

// Verdict-only check point (expanded pair test, early exit at frame granularity).
template <typename R, bool ARM, int MO, bool EARLY>
__device__ __forceinline__ void check_point_fast(const Geom<R>& G, const R* sm, const R (&q)[kMaxDof], R t,
                                                 bool& hit, unsigned& pairs) {
    const R* sph = sm;
    const R* way = sm + G.off_way;
    const R* vel = sm + G.off_vel;
    const R* rad = sm + G.off_rad;
    for (int m0 = 0; m0 < G.M; m0 += MO) {
        ObsTerms<R, MO> O;
#pragma unroll
        for (int j = 0; j < MO; ++j) {
            const int m = m0 + j;
            if (m < G.M) {
                R x, y, z;
                obstacle_at(way + 4 * G.K * m, vel + 4 * G.K * m, G.K, t, x, y, z);
                x -= G.ref[0];
                y -= G.ref[1];
                z -= G.ref[2];
                const R r = rad[m];
                O.ox[j] = R(-2) * x;
                O.oy[j] = R(-2) * y;
                O.oz[j] = R(-2) * z;
                O.ro[j] = R(-2) * r;
                O.B[j] = x * x + y * y + z * z - r * r;
            } else {
                O.ox[j] = O.oy[j] = O.oz[j] = O.ro[j] = R(0);
                O.B[j] = R(1e30);
            }
        }
        const unsigned real = (unsigned)min(MO, G.M - m0);
        if (!ARM) {
            const R px = q[0] - G.ref[0], py = q[1] - G.ref[1], pz = ((G.dof > 2) ? q[2] : R(0)) - G.ref[2];
            for (int s = 0; s < G.S; ++s) {
                if (sphere_hits<R, MO>(px + sph[4 * s], py + sph[4 * s + 1], pz + sph[4 * s + 2], sph[4 * s + 3], O))
                    hit = true;
            }
            pairs += real * (unsigned)G.S;
        } else {
            Frame<R> F;
            frame_identity(F);
            for (int j = 0; j <= G.dof; ++j) {
                if (j > 0) frame_step(F, G.a[j - 1], G.d[j - 1], G.ca[j - 1], G.sa[j - 1], q[j - 1] + G.th0[j - 1]);
                const R ox = F.o[0] - G.ref[0], oy = F.o[1] - G.ref[1], oz = F.o[2] - G.ref[2];
                for (int s = G.link_start[j]; s < G.link_start[j + 1]; ++s) {
                    const R px = sph[4 * s], py = sph[4 * s + 1], pz = sph[4 * s + 2];
                    const R cx = ox + px * F.X[0] + py * F.Y[0] + pz * F.Z[0];
                    const R cy = oy + px * F.X[1] + py * F.Y[1] + pz * F.Z[1];
                    const R cz = oz + px * F.X[2] + py * F.Y[2] + pz * F.Z[2];
                    if (sphere_hits<R, MO>(cx, cy, cz, sph[4 * s + 3], O)) hit = true;
                }
                pairs += real * (unsigned)(G.link_start[j + 1] - G.link_start[j]);
                if (EARLY && hit) break;
            }
        }
        if (EARLY && hit) break;
    }
}

// FP32 verdict path. Obstacle position at time t from the shared-memory
// tables: the segment index is the number of waypoint times t_1..t_{K-1} not
// after max(t, t_0) (times are strictly increasing; the table is +inf padded),
// then one waypoint and one velocity record are read as float4.
__device__ __forceinline__ void obstacle_at_f32(const float4* way, const float4* vel, const float4* tim, int K,
                                                float t, float& x, float& y, float& z) {
    const float tc = fmaxf(t, way[0].x);
    const float4 ta = tim[0];
    int k = (ta.x <= tc) + (ta.y <= tc) + (ta.z <= tc) + (ta.w <= tc);
    if (K > 5) {
        const float4 tb = tim[1];
        k += (tb.x <= tc) + (tb.y <= tc) + (tb.z <= tc) + (tb.w <= tc);
    }
    const float4 w = way[k];
    const float4 v = vel[k];
    const float dtk = tc - w.x;
    x = fmaf(dtk, v.x, w.y);
    y = fmaf(dtk, v.y, w.z);
    z = fmaf(dtk, v.z, w.w);
}

__device__ __forceinline__ float min3f(float a, float b, float c) {
    float r;
    asm("min.f32 %0, %1, %2, %3;" : "=f"(r) : "f"(a), "f"(b), "f"(c));
    return r;
}

// Packed obstacle terms of one chunk: lanes (2h, 2h+1) of obstacle pairs.
template <int MO>
struct ObsPacked {
    unsigned long long ox[MO / 2], oy[MO / 2], oz[MO / 2], ro[MO / 2], B[MO / 2];
};

// One robot sphere against a chunk: packed FMAs build
//   B_o + (-2 o).c [+ (-2 r_o) r_s]
// for two obstacles per instruction, three-input mins reduce them. With one
// obstacle radius R_o for all obstacles (UNI) the r_s r_o cross term is
// per-sphere and moves into the threshold r_s (r_s + 2 R_o) - |c|^2.
template <int MO, bool UNI>
__device__ __forceinline__ bool sphere_hits_packed(float cx, float cy, float cz, float rs, float ro_uni,
                                                   const ObsPacked<MO>& O) {
    const float thr = rs * (UNI ? rs + 2.f * ro_uni : rs) - (cx * cx + cy * cy + cz * cz);
    const unsigned long long CX = pk2(cx, cx), CY = pk2(cy, cy), CZ = pk2(cz, cz);
    const unsigned long long RS = UNI ? 0ull : pk2(rs, rs);
    float m0 = rinf<float>(), m1 = rinf<float>();
#pragma unroll
    for (int h = 0; h < MO / 2; ++h) {
        unsigned long long a = ffma2(CX, O.ox[h], O.B[h]);
        a = ffma2(CY, O.oy[h], a);
        a = ffma2(CZ, O.oz[h], a);
        if (!UNI) a = ffma2(RS, O.ro[h], a);
        float lo, hi;
        upk2(a, lo, hi);
        if (h & 1) m1 = min3f(m1, lo, hi);
        else m0 = min3f(m0, lo, hi);
    }
    return fminf(m0, m1) < thr;
}

template <bool ARM, int MO, bool EARLY, bool UNI>
__device__ __forceinline__ void check_point_f32(const Geom<float>& G, const float* sm, const float (&q)[kMaxDof],
                                                float t, bool& hit, unsigned& pairs) {
    const float4* sph = reinterpret_cast<const float4*>(sm);
    const float4* way = reinterpret_cast<const float4*>(sm + G.off_way);
    const float4* vel = reinterpret_cast<const float4*>(sm + G.off_vel);
    const float4* tim = reinterpret_cast<const float4*>(sm + G.off_tim);
    const float* rad = sm + G.off_rad;
    const float ro_uni = G.ro_uni;
    for (int m0 = 0; m0 < G.M; m0 += MO) {
        ObsPacked<MO> O;
#pragma unroll
        for (int h = 0; h < MO / 2; ++h) {
            float x[2], y[2], z[2], r[2], b[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
                const int m = m0 + 2 * h + u;
                if (m < G.M) {
                    obstacle_at_f32(way + G.K * m, vel + G.K * m, tim + 2 * m, G.K, t, x[u], y[u], z[u]);
                    if (!ARM) {
                        x[u] -= G.ref[0];
                        y[u] -= G.ref[1];
                        z[u] -= G.ref[2];
                    }
                    r[u] = UNI ? ro_uni : rad[m];
                    b[u] = x[u] * x[u] + y[u] * y[u] + z[u] * z[u] - r[u] * r[u];
                } else {
                    x[u] = y[u] = z[u] = r[u] = 0.f;
                    b[u] = 1e30f;
                }
            }
            O.ox[h] = pk2(-2.f * x[0], -2.f * x[1]);
            O.oy[h] = pk2(-2.f * y[0], -2.f * y[1]);
            O.oz[h] = pk2(-2.f * z[0], -2.f * z[1]);
            O.ro[h] = pk2(-2.f * r[0], -2.f * r[1]);
            O.B[h] = pk2(b[0], b[1]);
        }
        const unsigned real = (unsigned)min(MO, G.M - m0);
        if (!ARM) {
            const float px = q[0] - G.ref[0], py = q[1] - G.ref[1], pz = ((G.dof > 2) ? q[2] : 0.f) - G.ref[2];
            for (int s = 0; s < G.S; ++s) {
                const float4 sp = sph[s];
                if (sphere_hits_packed<MO, UNI>(px + sp.x, py + sp.y, pz + sp.z, sp.w, ro_uni, O)) hit = true;
            }
            pairs += real * (unsigned)G.S;
        } else {
            Frame<float> F;
            frame_identity(F);
            for (int j = 0; j <= G.dof; ++j) {
                if (j > 0) frame_step(F, G.a[j - 1], G.d[j - 1], G.ca[j - 1], G.sa[j - 1], q[j - 1] + G.th0[j - 1]);
                const float ox = F.o[0], oy = F.o[1], oz = F.o[2];
                const int s0 = G.link_start[j], s1 = G.link_start[j + 1];
                int s = s0;
                for (; s + 1 < s1; s += 2) {
                    const float4 sp = sph[s];
                    const float4 sq = sph[s + 1];
                    const float cx = ox + sp.x * F.X[0] + sp.y * F.Y[0] + sp.z * F.Z[0];
                    const float cy = oy + sp.x * F.X[1] + sp.y * F.Y[1] + sp.z * F.Z[1];
                    const float cz = oz + sp.x * F.X[2] + sp.y * F.Y[2] + sp.z * F.Z[2];
                    const float dx = ox + sq.x * F.X[0] + sq.y * F.Y[0] + sq.z * F.Z[0];
                    const float dy = oy + sq.x * F.X[1] + sq.y * F.Y[1] + sq.z * F.Z[1];
                    const float dz = oz + sq.x * F.X[2] + sq.y * F.Y[2] + sq.z * F.Z[2];
                    const bool h0 = sphere_hits_packed<MO, UNI>(cx, cy, cz, sp.w, ro_uni, O);
                    const bool h1 = sphere_hits_packed<MO, UNI>(dx, dy, dz, sq.w, ro_uni, O);
                    hit = hit | h0 | h1;
                }
                if (s < s1) {
                    const float4 sp = sph[s];
                    const float cx = ox + sp.x * F.X[0] + sp.y * F.Y[0] + sp.z * F.Z[0];
                    const float cy = oy + sp.x * F.X[1] + sp.y * F.Y[1] + sp.z * F.Z[1];
                    const float cz = oz + sp.x * F.X[2] + sp.y * F.Y[2] + sp.z * F.Z[2];
                    hit = hit | sphere_hits_packed<MO, UNI>(cx, cy, cz, sp.w, ro_uni, O);
                }
                pairs += real * (unsigned)(s1 - s0);
                if (EARLY && hit) break;
            }
        }
        if (EARLY && hit) break;
    }
}

template <typename R, bool ARM, int MO, bool CLEAR, bool EARLY>
__device__ __forceinline__ void check_point(const Geom<R>& G, const R* sm, const R (&q)[kMaxDof], R t, bool& hit,
                                            R& clr, unsigned& pairs) {
    if (!CLEAR) {
        if constexpr (sizeof(R) == 4 && MO % 2 == 0) {
            if (G.uniform_ro) check_point_f32<ARM, MO, EARLY, true>(G, sm, q, t, hit, pairs);
            else check_point_f32<ARM, MO, EARLY, false>(G, sm, q, t, hit, pairs);
        } else {
            check_point_fast<R, ARM, MO, EARLY>(G, sm, q, t, hit, pairs);
        }
        return;
    }
    const R* sph = sm;
    const R* way = sm + G.off_way;
    const R* vel = sm + G.off_vel;
    const R* rad = sm + G.off_rad;
    for (int m0 = 0; m0 < G.M; m0 += MO) {
        R ox[MO], oy[MO], oz[MO], orr[MO];
#pragma unroll
        for (int j = 0; j < MO; ++j) {
            int m = m0 + j;
            if (m < G.M) {
                obstacle_at(way + 4 * G.K * m, vel + 4 * G.K * m, G.K, t, ox[j], oy[j], oz[j]);
                orr[j] = rad[m];
            } else {
                ox[j] = oy[j] = oz[j] = R(1e18);
                orr[j] = R(0);
            }
        }
        const unsigned real = (unsigned)min(MO, G.M - m0);
        if (!ARM) {
            R px = q[0], py = q[1], pz = (G.dof > 2) ? q[2] : R(0);
            for (int s = 0; s < G.S; ++s) {
                test_sphere<R, MO, CLEAR>(px + sph[4 * s], py + sph[4 * s + 1], pz + sph[4 * s + 2], sph[4 * s + 3],
                                          ox, oy, oz, orr, hit, clr);
            }
            pairs += real * (unsigned)G.S;
        } else {
            Frame<R> F;
            frame_identity(F);
            for (int j = 0; j <= G.dof; ++j) {
                if (j > 0) frame_step(F, G.a[j - 1], G.d[j - 1], G.ca[j - 1], G.sa[j - 1], q[j - 1] + G.th0[j - 1]);
                for (int s = G.link_start[j]; s < G.link_start[j + 1]; ++s) {
                    R px = sph[4 * s], py = sph[4 * s + 1], pz = sph[4 * s + 2];
                    R cx = F.o[0] + px * F.X[0] + py * F.Y[0] + pz * F.Z[0];
                    R cy = F.o[1] + px * F.X[1] + py * F.Y[1] + pz * F.Z[1];
                    R cz = F.o[2] + px * F.X[2] + py * F.Y[2] + pz * F.Z[2];
                    test_sphere<R, MO, CLEAR>(cx, cy, cz, sph[4 * s + 3], ox, oy, oz, orr, hit, clr);
                }
                pairs += real * (unsigned)(G.link_start[j + 1] - G.link_start[j]);
                if (EARLY && !CLEAR && hit) break;
            }
        }
        if (EARLY && !CLEAR && hit) break;
    }
}

// Self-collision of an arm state (optional): FK into a lane-private table of
// sphere centres, then the sphere predicate on the problem's pair list (pairs
// on frames at least two apart that do not touch at q = 0), read from the
// geometry blob in shared memory as a * 64 + b.
template <typename R, bool CLEAR>
__device__ __noinline__ void self_check(const Geom<R>& G, const R* sm, const R (&q)[kMaxDof], bool& hit, R& clr) {
    R c[kMaxSpheres][3];
    const R* sph = sm;
    Frame<R> F;
    frame_identity(F);
    for (int j = 0; j <= G.dof; ++j) {
        if (j > 0) frame_step(F, G.a[j - 1], G.d[j - 1], G.ca[j - 1], G.sa[j - 1], q[j - 1] + G.th0[j - 1]);
        for (int s = G.link_start[j]; s < G.link_start[j + 1]; ++s) {
            const R px = sph[4 * s], py = sph[4 * s + 1], pz = sph[4 * s + 2];
            for (int i = 0; i < 3; ++i) c[s][i] = F.o[i] + px * F.X[i] + py * F.Y[i] + pz * F.Z[i];
        }
    }
    const R* pairs = sm + G.off_self;
    for (int k = 0; k < G.n_self; ++k) {
        const int code = (int)pairs[k];
        const int a = code >> 6, b = code & 63;
        const R dx = c[a][0] - c[b][0], dy = c[a][1] - c[b][1], dz = c[a][2] - c[b][2];
        const R d2 = dx * dx + dy * dy + dz * dz;
        const R rr = sph[4 * a + 3] + sph[4 * b + 3];
        if (d2 < rr * rr) {
            hit = true;
            if (!CLEAR) return;
        }
        if (CLEAR) {
            const R cl = rsqrt_r(d2) - rr;
            clr = cl < clr ? cl : clr;
        }
    }
}

template <typename R>
__device__ __forceinline__ void atomic_min_r(R* addr, R v);
template <>
__device__ __forceinline__ void atomic_min_r<float>(float* addr, float v) {
    atomicMin(reinterpret_cast<int*>(addr), ord_enc(v));
}
template <>
__device__ __forceinline__ void atomic_min_r<double>(double* addr, double v) {
    atomicMin(reinterpret_cast<long long*>(addr), ord_enc(v));
}

// Exclusive block scan (all threads participate).
__device__ __forceinline__ int block_scan_excl(int v, int* sh, int* total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int x = v;
    for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        const int nw = blockDim.x >> 5;
        int y = lane < nw ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int z = __shfl_up_sync(0xffffffffu, y, o);
            if (lane >= o) y += z;
        }
        if (lane < nw) sh[lane] = y;
    }
    __syncthreads();
    const int before = (warp > 0 ? sh[warp - 1] : 0) + x - v;
    *total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before;
}

// Edges per shared-memory window in the large-batch mode.
constexpr int kWin = 64;

// Kernel body: G and E may live in registers/parameters (single problem) or in
// shared memory (batch); smem_raw is the dynamic shared-memory buffer.
// cta / ncta: this CTA's index among the CTAs sharing the batch. staged: the
// geometry blob is already in shared memory at smem_raw (persistent kernel);
// otherwise one TMA bulk copy stages it.
template <typename R, bool ARM, int MO, bool CLEAR, bool EARLY>
__device__ __forceinline__ void validate_body(const Geom<R>& G, const EdgeBatch<R>& E, unsigned char* smem_raw,
                                              int cta, int ncta, bool staged = false) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int scan_sh[32];
    R* sm = reinterpret_cast<R*>(smem_raw);
    const int n = E.n_dev ? *E.n_dev : E.n_host;
    if (n <= 0 || (E.done && *E.done)) return;
    if (!staged) {
        if (threadIdx.x == 0) mbar_init(&bar, 1);
        __syncthreads();
        if (threadIdx.x == 0) {
            mbar_expect_tx(&bar, G.blob_bytes);
            bulk_g2s(sm, G.blob, G.blob_bytes, &bar);
        }
    }
    // Without precomputed offsets every CTA scans the (small) count array
    // into shared memory while the geometry copy is in flight. Every CTA must
    // derive the same offsets: the remaining-points pass (phase 2) skips the
    // edges the coarse pass found hit (flag bit 0, written by the previous
    // launch) and marks its own hits with 2, so flags set while other CTAs
    // are still scanning never change a count.
    int* soff = reinterpret_cast<int*>(smem_raw + G.blob_bytes);
    if (!E.off) {
        const int per = (n + blockDim.x - 1) / blockDim.x;
        const int i0 = threadIdx.x * per, i1 = min(n, i0 + per);
        auto eff = [&](int i) -> int {
            const int c = E.cnt[i];
            if (E.phase == 1) return (c + 7) >> 3;
            if (E.phase == 2) return (E.hit[i] & 1) ? 0 : c;
            return c;
        };
        constexpr int kStage = 8;  // counts a thread keeps in registers
        int cv[kStage];
        int sum = 0;
        if (per <= kStage) {
            // One round of independent loads.
#pragma unroll
            for (int k = 0; k < kStage; ++k) cv[k] = i0 + k < i1 ? eff(i0 + k) : 0;
#pragma unroll
            for (int k = 0; k < kStage; ++k) sum += cv[k];
        } else {
            for (int i = i0; i < i1; ++i) sum += eff(i);
        }
        int tot;
        int pre = block_scan_excl(sum, scan_sh, &tot);
        if (per <= kStage) {
#pragma unroll
            for (int k = 0; k < kStage; ++k) {
                if (i0 + k < i1) soff[i0 + k] = pre;
                pre += cv[k];
            }
        } else {
            for (int i = i0; i < i1; ++i) {
                soff[i] = pre;
                pre += eff(i);
            }
        }
        if (threadIdx.x == 0) soff[n] = tot;
        __syncthreads();
    }
    if (!staged && !mbar_wait(&bar, 0)) {
        if (threadIdx.x == 0 && E.err) atomicOr(E.err, kErrTimeout);
        return;
    }
    auto off_at = [&](int e) -> long long { return E.off ? E.off[e] : (long long)soff[e]; };

    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    const int wpb = blockDim.x >> 5;
    unsigned long long done = 0, pairs_total = 0;

    // One check point g of edge e: interpolate, run FK and the pair tests.
    auto process = [&](long long g, int e, long long e_off) {
        if (EARLY && !CLEAR) {
            if (*(volatile int*)(E.hit + e)) return;
        }
        const int c = E.cnt[e];
        int jj = (int)(g - e_off) + 1;
        if (E.phase == 1) {
            const int c0 = (c + 7) >> 3;
            jj = (int)(((long long)jj * c + c0 - 1) / c0);
        }
        const R s = R(jj) / R(c);
        const R* qa = E.qa + (size_t)e * E.qstride;
        const R* qb = E.qb + (size_t)e * E.qstride;
        R q[kMaxDof];
        bool hit = false;
#pragma unroll
        for (int i = 0; i < kMaxDof; ++i) {
            if (i < G.dof) {
                q[i] = qa[i] + s * (qb[i] - qa[i]);
                hit = hit || (q[i] < G.qlo[i]) || (q[i] > G.qhi[i]);
            } else {
                q[i] = R(0);
            }
        }
        const R ta = E.ta[e];
        const R t = ta + s * (E.tb[e] - ta);
        R clr = rinf<R>();
        unsigned pairs = 0;
        if (ARM) check_point<R, true, MO, CLEAR, EARLY>(G, sm, q, t, hit, clr, pairs);
        else check_point<R, false, MO, CLEAR, EARLY>(G, sm, q, t, hit, clr, pairs);
        if (ARM && G.n_self > 0 && (CLEAR || !hit)) self_check<R, CLEAR>(G, sm, q, hit, clr);
        if (hit) E.hit[e] = E.phase == 2 ? 2 : 1;
        if (CLEAR) atomic_min_r<R>(E.clear + e, clr);
        ++done;
        pairs_total += pairs;
    };

    if (!E.off) {
        // Small batches (offsets scanned into shared memory): the flat range of
        // check points is cut into 32-point groups dealt round-robin over the
        // CTAs first (group k to CTA k mod grid), so that a batch smaller than
        // the resident grid still spreads over every SM; each lane finds its
        // edge by binary search in shared memory.
        const long long total = soff[n];
        const long long ngroups = (total + 31) >> 5;
        const long long gstride = (long long)ncta * wpb;
        for (long long k = (long long)warp * ncta + cta; k < ngroups; k += gstride) {
            const long long g = k * 32 + lane;
            if (g >= total) continue;
            int lo = 0, hi = n - 1;
            while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (soff[mid] <= g) lo = mid;
                else hi = mid - 1;
            }
            process(g, lo, soff[lo]);
        }
    } else {
        // Large batches (precomputed offsets in global memory): CTAs take
        // windows of kWin consecutive edges (from the window counter as they
        // finish the previous one, so the batch ends within one window of
        // balance; or round-robin without a counter), stage the window's
        // offsets in shared memory and spread its check points over their warps.
        long long* woff = reinterpret_cast<long long*>(smem_raw + G.blob_bytes);
        __shared__ int s_win;
        for (int k = 0;; ++k) {
            __syncthreads();   // the previous window's offsets are no longer read
            if (threadIdx.x == 0) s_win = E.win_next ? atomicAdd(E.win_next, 1) : cta + k * ncta;
            __syncthreads();
            if (s_win >= (n + kWin - 1) / kWin) break;
            const int w0 = s_win * kWin;
            const int wn = min(kWin, n - w0);
            for (int i = threadIdx.x; i <= wn; i += blockDim.x) woff[i] = E.off[w0 + i];
            __syncthreads();
            const long long ob = woff[0], oe = woff[wn];
            for (long long g = ob + warp * 32 + lane; g < oe; g += wpb * 32) {
                int lo = 0, hi = wn - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (woff[mid] <= g) lo = mid;
                    else hi = mid - 1;
                }
                process(g, w0 + lo, woff[lo]);
            }
        }
    }
    if (E.points_done) {
        for (int o = 16; o > 0; o >>= 1) done += __shfl_xor_sync(0xffffffffu, done, o);
        if (lane == 0 && done) atomicAdd(E.points_done, done);
    }
    if (E.pairs_done) {
        for (int o = 16; o > 0; o >>= 1) pairs_total += __shfl_xor_sync(0xffffffffu, pairs_total, o);
        if (lane == 0 && pairs_total) atomicAdd(E.pairs_done, pairs_total);
    }
}

}  // namespace stp
