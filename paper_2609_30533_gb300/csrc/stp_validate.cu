// Edge validation kernel (collision checking of space-time edges against
// moving obstacles; Sec. "Simulation Protocol": obstacle positions are
// interpolated at each absolute query time) and the flat-batch helpers.
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
constexpr int kWin = 256;

// Kernel body: G and E may live in registers/parameters (single problem) or in
// shared memory (batch); smem_raw is the dynamic shared-memory buffer.
template <typename R, bool ARM, int MO, bool CLEAR, bool EARLY>
__device__ __forceinline__ void validate_body(const Geom<R>& G, const EdgeBatch<R>& E, unsigned char* smem_raw) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int scan_sh[32];
    R* sm = reinterpret_cast<R*>(smem_raw);
    const int n = E.n_dev ? *E.n_dev : E.n_host;
    if (n <= 0 || (E.done && *E.done)) return;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_expect_tx(&bar, G.blob_bytes);
        bulk_g2s(sm, G.blob, G.blob_bytes, &bar);
    }
    // Without precomputed offsets every CTA scans the (small) count array
    // into shared memory while the geometry copy is in flight.
    int* soff = reinterpret_cast<int*>(smem_raw + G.blob_bytes);
    if (!E.off) {
        const int per = (n + blockDim.x - 1) / blockDim.x;
        const int i0 = threadIdx.x * per, i1 = min(n, i0 + per);
        auto eff = [&](int i) -> int {
            const int c = E.cnt[i];
            if (E.phase == 1) return (c + 7) >> 3;
            if (E.phase == 2) return E.hit[i] ? 0 : c;
            return c;
        };
        int sum = 0;
        for (int i = i0; i < i1; ++i) sum += eff(i);
        int tot;
        int pre = block_scan_excl(sum, scan_sh, &tot);
        for (int i = i0; i < i1; ++i) {
            soff[i] = pre;
            pre += eff(i);
        }
        if (threadIdx.x == 0) soff[n] = tot;
        __syncthreads();
    }
    if (!mbar_wait(&bar, 0)) {
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
        if (hit) E.hit[e] = 1;
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
        const long long gstride = (long long)gridDim.x * wpb;
        for (long long k = (long long)warp * gridDim.x + blockIdx.x; k < ngroups; k += gstride) {
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
        // windows of kWin consecutive edges, stage the window's offsets in
        // shared memory and spread its check points over their warps.
        long long* woff = reinterpret_cast<long long*>(smem_raw + G.blob_bytes);
        for (int w0 = blockIdx.x * kWin; w0 < n; w0 += gridDim.x * kWin) {
            const int wn = min(kWin, n - w0);
            __syncthreads();
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

template <typename R, bool ARM, int MO, bool CLEAR, bool EARLY>
__global__ void __launch_bounds__(256, (sizeof(R) == 4 && MO <= 16) ? 2 : 1) k_validate(Geom<R> G, EdgeBatch<R> E) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    validate_body<R, ARM, MO, CLEAR, EARLY>(G, E, smem_raw);
}

// Batched planner form: problem blockIdx.y; its geometry and state are staged
// in shared memory, its extension (which = 0) or bridge (which = 1) edge
// entries are validated; arm vs point robot is chosen per problem.
template <typename R, int MO>
__global__ void __launch_bounds__(256, (sizeof(R) == 4 && MO <= 16) ? 2 : 1)
    k_validate_batch(const Geom<R>* __restrict__ Gs, const State<R>* __restrict__ Ss, int which) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Geom<R> G;
    __shared__ State<R> S;
    stage_problem(Gs, Ss, blockIdx.y, G, S);
    EdgeBatch<R> E = which == 0 ? ext_batch(S) : bridge_batch(S);
    E.phase = which >= 1 ? which : 0;   // which 1: coarse bridge pass, 2: remaining bridge points
    if (G.arm) validate_body<R, true, MO, false, true>(G, E, smem_raw);
    else validate_body<R, false, MO, false, true>(G, E, smem_raw);
}

// ---------------------------------------------------------------------------
// Host launchers.
// ---------------------------------------------------------------------------
static int g_num_sms = 0;

int validate_grid_blocks() {
    if (g_num_sms == 0) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&g_num_sms, cudaDevAttrMultiProcessorCount, dev);
        if (g_num_sms <= 0) g_num_sms = 1;
    }
    return g_num_sms;
}

template <typename R, bool ARM, int MO, bool CLEAR, bool EARLY>
static cudaError_t launch_v(const Geom<R>& g, const EdgeBatch<R>& e, int grid_blocks, cudaStream_t st) {
    auto kern = k_validate<R, ARM, MO, CLEAR, EARLY>;
    static int configured_bytes = -1;
    static int blocks_per_sm = 0;
    int smem = (int)g.blob_bytes + (e.off ? (int)(sizeof(long long) * (kWin + 1))
                                          : (int)(sizeof(int) * (e.n_host + 1)));
    if (smem > configured_bytes) {
        cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
        if (err != cudaSuccess) return err;
        configured_bytes = smem;
        blocks_per_sm = 0;
    }
    if (blocks_per_sm == 0) {
        cudaError_t err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks_per_sm, kern, 256, smem);
        if (err != cudaSuccess) return err;
        if (blocks_per_sm < 1) blocks_per_sm = 1;
    }
    int grid = grid_blocks > 0 ? grid_blocks : validate_grid_blocks() * blocks_per_sm;
    kern<<<grid, 256, smem, st>>>(g, e);
    return cudaGetLastError();
}

template <typename R, bool ARM, bool CLEAR, bool EARLY>
static cudaError_t launch_mo(const Geom<R>& g, const EdgeBatch<R>& e, int grid_blocks, cudaStream_t st) {
    if (CLEAR) return launch_v<R, ARM, 16, CLEAR, EARLY>(g, e, grid_blocks, st);
    if (g.M <= 8) return launch_v<R, ARM, 8, CLEAR, EARLY>(g, e, grid_blocks, st);
    if (g.M <= 16) return launch_v<R, ARM, 16, CLEAR, EARLY>(g, e, grid_blocks, st);
    return launch_v<R, ARM, 32, CLEAR, EARLY>(g, e, grid_blocks, st);
}

// ---------------------------------------------------------------------------
// Closed-form (continuous) validation of point-robot edges, one lane per
// edge. Between consecutive breakpoints (the edge's end times and each
// obstacle waypoint time inside them) a robot sphere and an obstacle both
// move linearly, so their difference runs along the segment from d(t0) to
// d(t1) and its smallest norm is the distance from the origin to that segment.
// A pair collides iff that squared minimum < (r + r_o)^2; the edge stays in
// the convex configuration box iff both ends do.
// ---------------------------------------------------------------------------
template <typename R, bool CLEAR>
__global__ void __launch_bounds__(256) k_validate_cont(Geom<R> G, EdgeBatch<R> E) {
    const int n = E.n_dev ? *E.n_dev : E.n_host;
    if (n <= 0 || (E.done && *E.done)) return;
    const R* sph = G.blob;
    const R* way = G.blob + G.off_way;
    const R* vel = G.blob + G.off_vel;
    const R* rad = G.blob + G.off_rad;
    unsigned long long done = 0, pairs_total = 0;
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
        if (E.cnt[e] <= 0) continue;
        const R* qa = E.qa + (size_t)e * E.qstride;
        const R* qb = E.qb + (size_t)e * E.qstride;
        const R ta = E.ta[e], tb = E.tb[e];
        bool hit = false;
        for (int j = 0; j < G.dof; ++j)
            hit = hit || qa[j] < G.qlo[j] || qa[j] > G.qhi[j] || qb[j] < G.qlo[j] || qb[j] > G.qhi[j];
        const R pa[3] = {qa[0], qa[1], G.dof > 2 ? qa[2] : R(0)};
        const R pb[3] = {qb[0], qb[1], G.dof > 2 ? qb[2] : R(0)};
        R clr = rinf<R>();
        for (int m = 0; m < G.M; ++m) {
            const R* W = way + 4 * G.K * m;
            const R* V = vel + 4 * G.K * m;
            const R ro = rad[m];
            R t0 = ta;
            for (int k = 0; k <= G.K; ++k) {
                // next breakpoint: waypoint k if inside (ta, tb), the end at k == K
                R t1;
                if (k < G.K) {
                    t1 = W[4 * k];
                    if (!(t1 > ta && t1 < tb)) continue;
                } else {
                    t1 = tb;
                }
                const R f0 = tb > ta ? (t0 - ta) / (tb - ta) : R(0);
                const R f1 = tb > ta ? (t1 - ta) / (tb - ta) : R(0);
                R o0[3], o1[3];
                obstacle_at(W, V, G.K, t0, o0[0], o0[1], o0[2]);
                obstacle_at(W, V, G.K, t1, o1[0], o1[1], o1[2]);
                for (int sp = 0; sp < G.S; ++sp) {
                    R d0[3], w[3];
                    for (int i = 0; i < 3; ++i) {
                        const R c0 = (pa[i] + f0 * (pb[i] - pa[i])) + sph[4 * sp + i];
                        const R c1 = (pa[i] + f1 * (pb[i] - pa[i])) + sph[4 * sp + i];
                        d0[i] = c0 - o0[i];
                        w[i] = (c1 - o1[i]) - d0[i];
                    }
                    const R a = w[0] * w[0] + w[1] * w[1] + w[2] * w[2];
                    const R b = d0[0] * w[0] + d0[1] * w[1] + d0[2] * w[2];
                    R u = a > R(0) ? -b / a : R(0);
                    u = u < R(0) ? R(0) : (u > R(1) ? R(1) : u);
                    R d2 = R(0);
                    for (int i = 0; i < 3; ++i) {
                        const R x = d0[i] + u * w[i];
                        d2 += x * x;
                    }
                    const R rr = sph[4 * sp + 3] + ro;
                    hit = hit || (d2 < rr * rr);
                    if (CLEAR) {
                        const R cl = rsqrt_r(d2) - rr;
                        clr = cl < clr ? cl : clr;
                    }
                }
                pairs_total += (unsigned long long)G.S;
                t0 = t1;
            }
        }
        E.hit[e] = hit ? 1 : 0;
        if (CLEAR) atomic_min_r<R>(E.clear + e, clr);  // order-encoded like the discrete path
        ++done;
    }
    const int lane = threadIdx.x & 31;
    if (E.points_done) {
        for (int o = 16; o > 0; o >>= 1) done += __shfl_xor_sync(0xffffffffu, done, o);
        if (lane == 0 && done) atomicAdd(E.points_done, done);
    }
    if (E.pairs_done) {
        for (int o = 16; o > 0; o >>= 1) pairs_total += __shfl_xor_sync(0xffffffffu, pairs_total, o);
        if (lane == 0 && pairs_total) atomicAdd(E.pairs_done, pairs_total);
    }
}

template <typename R>
cudaError_t launch_validate(const Geom<R>& g, const EdgeBatch<R>& e, bool clearance, bool early_exit,
                            int grid_blocks, cudaStream_t st) {
    if (g.continuous) {
        const int blocks = grid_blocks > 0 ? grid_blocks : validate_grid_blocks() * 2;
        if (clearance) k_validate_cont<R, true><<<blocks, 256, 0, st>>>(g, e);
        else k_validate_cont<R, false><<<blocks, 256, 0, st>>>(g, e);
        return cudaGetLastError();
    }
    if (g.arm) {
        if (clearance) return launch_mo<R, true, true, false>(g, e, grid_blocks, st);
        if (early_exit) return launch_mo<R, true, false, true>(g, e, grid_blocks, st);
        return launch_mo<R, true, false, false>(g, e, grid_blocks, st);
    }
    if (clearance) return launch_mo<R, false, true, false>(g, e, grid_blocks, st);
    if (early_exit) return launch_mo<R, false, false, true>(g, e, grid_blocks, st);
    return launch_mo<R, false, false, false>(g, e, grid_blocks, st);
}

template <typename R, int MO>
static cudaError_t launch_vb(const Geom<R>* Gs, const State<R>* Ss, int P, int which, int ctas_per_problem,
                             int smem_bytes, cudaStream_t st) {
    auto kern = k_validate_batch<R, MO>;
    static int configured = -1;
    if (smem_bytes > configured) {
        cudaError_t err = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
        if (err != cudaSuccess) return err;
        configured = smem_bytes;
    }
    if (P <= 0) return cudaSuccess;  // configuration only
    kern<<<dim3(ctas_per_problem, P), 256, smem_bytes, st>>>(Gs, Ss, which);
    return cudaGetLastError();
}

// P <= 0 only sets the kernel's shared-memory attribute (nothing is launched).
template <typename R>
cudaError_t launch_validate_batch(const Geom<R>* Gs, const State<R>* Ss, int P, int which, int max_obs,
                                  int ctas_per_problem, int smem_bytes, cudaStream_t st) {
    if (max_obs <= 8) return launch_vb<R, 8>(Gs, Ss, P, which, ctas_per_problem, smem_bytes, st);
    return launch_vb<R, 16>(Gs, Ss, P, which, ctas_per_problem, smem_bytes, st);
}
template cudaError_t launch_validate_batch<float>(const Geom<float>*, const State<float>*, int, int, int, int, int,
                                                  cudaStream_t);

// Check-point counts, c = max(1, ceil(max(D, v_max |dt|) / res - 1e-3)),
// evaluated in double from the stored endpoints.
template <typename R>
__global__ void k_edge_counts(double vmax, int dof, const R* qa, const R* ta, const R* qb, const R* tb, int qstride,
                              int n, double res, int* cnt) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    double s2 = 0.0;
    for (int i = 0; i < dof; ++i) {
        double dd = (double)qb[(size_t)e * qstride + i] - (double)qa[(size_t)e * qstride + i];
        s2 = __dadd_rn(s2, __dmul_rn(dd, dd));
    }
    double D = sqrt(s2);
    double L = fmax(D, __dmul_rn(vmax, fabs((double)tb[e] - (double)ta[e])));
    double c = ceil(L / res - 1e-3);
    cnt[e] = c < 1.0 ? 1 : (int)c;
}

template <typename R>
cudaError_t launch_edge_counts(const Geom<R>& g, const R* qa, const R* ta, const R* qb, const R* tb, int qstride,
                               int n, double res, int* cnt, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_edge_counts<R><<<(n + 255) / 256, 256, 0, st>>>(g.vmax_d, g.dof, qa, ta, qb, tb, qstride, n, res, cnt);
    return cudaGetLastError();
}

// Exclusive prefix sum of counts into off[0..n] (off[n] = total); three phases.
constexpr int kScanBlock = 1024;
constexpr int kScanPer = 4;
constexpr int kScanTile = kScanBlock * kScanPer;

__device__ __forceinline__ long long block_exclusive_scan(long long v, long long* sh, long long* total) {
    // Warp scan then scan of warp totals.
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long x = v;
    for (int o = 1; o < 32; o <<= 1) {
        long long y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) sh[warp] = x;
    __syncthreads();
    if (warp == 0) {
        int nw = blockDim.x >> 5;
        long long w = lane < nw ? sh[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, w, o);
            if (lane >= o) w += y;
        }
        if (lane < nw) sh[lane] = w;
    }
    __syncthreads();
    long long before = (warp > 0 ? sh[warp - 1] : 0) + x - v;
    if (total) *total = sh[(blockDim.x >> 5) - 1];
    __syncthreads();
    return before;
}

__global__ void k_scan_tiles(const int* cnt, int n, long long* off, long long* tile_tot) {
    __shared__ long long sh[32];
    const int base = blockIdx.x * kScanTile + threadIdx.x * kScanPer;
    long long v[kScanPer];
    long long sum = 0;
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        v[i] = (base + i < n) ? cnt[base + i] : 0;
        sum += v[i];
    }
    long long tot;
    long long pre = block_exclusive_scan(sum, sh, &tot);
#pragma unroll
    for (int i = 0; i < kScanPer; ++i) {
        if (base + i < n) off[base + i] = pre;
        pre += v[i];
    }
    if (threadIdx.x == 0) tile_tot[blockIdx.x] = tot;
}

__global__ void k_scan_tops(long long* tile_tot, int ntiles, long long* off, int n) {
    __shared__ long long sh[32];
    long long carry = 0;
    for (int b0 = 0; b0 < ntiles; b0 += blockDim.x) {
        int b = b0 + threadIdx.x;
        long long v = b < ntiles ? tile_tot[b] : 0;
        long long tot;
        long long pre = block_exclusive_scan(v, sh, &tot);
        if (b < ntiles) tile_tot[b] = carry + pre;
        carry += tot;
    }
    if (threadIdx.x == 0) off[n] = carry;
}

__global__ void k_scan_add(long long* off, int n, const long long* tile_tot) {
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) off[i] += tile_tot[i / kScanTile];
}

cudaError_t launch_scan_counts(const int* cnt, int n, long long* off, long long* tile_tmp, cudaStream_t st) {
    if (n <= 0) {
        return cudaMemsetAsync(off, 0, sizeof(long long), st);
    }
    int ntiles = (n + kScanTile - 1) / kScanTile;
    k_scan_tiles<<<ntiles, kScanBlock, 0, st>>>(cnt, n, off, tile_tmp);
    k_scan_tops<<<1, kScanBlock, 0, st>>>(tile_tmp, ntiles, off, n);
    k_scan_add<<<(n + 255) / 256, 256, 0, st>>>(off, n, tile_tmp);
    return cudaGetLastError();
}

// Small fills and conversions used by the batch entry point.
__global__ void k_fill_u32(unsigned* p, long long n, unsigned v) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}
__global__ void k_fill_u64(unsigned long long* p, long long n, unsigned long long v) {
    long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) p[i] = v;
}
cudaError_t launch_fill(void* p, long long n, int bytes, unsigned long long v, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    int grid = (int)((n + 255) / 256);
    if (bytes == 4) k_fill_u32<<<grid, 256, 0, st>>>((unsigned*)p, n, (unsigned)v);
    else k_fill_u64<<<grid, 256, 0, st>>>((unsigned long long*)p, n, v);
    return cudaGetLastError();
}

template <typename R>
__global__ void k_finish_batch(int n, const int* hit, unsigned char* verdict, R* clear) {
    int e = blockIdx.x * blockDim.x + threadIdx.x;
    if (e >= n) return;
    verdict[e] = hit[e] ? 0 : 1;
    if (clear) clear[e] = ord_dec(*reinterpret_cast<const decltype(ord_enc(R(0)))*>(clear + e));
}
template <typename R>
cudaError_t launch_finish_batch(int n, const int* hit, unsigned char* verdict, R* clear, cudaStream_t st) {
    if (n <= 0) return cudaSuccess;
    k_finish_batch<R><<<(n + 255) / 256, 256, 0, st>>>(n, hit, verdict, clear);
    return cudaGetLastError();
}
template cudaError_t launch_finish_batch<float>(int, const int*, unsigned char*, float*, cudaStream_t);
template cudaError_t launch_finish_batch<double>(int, const int*, unsigned char*, double*, cudaStream_t);

template cudaError_t launch_validate<float>(const Geom<float>&, const EdgeBatch<float>&, bool, bool, int,
                                            cudaStream_t);
template cudaError_t launch_validate<double>(const Geom<double>&, const EdgeBatch<double>&, bool, bool, int,
                                             cudaStream_t);
template cudaError_t launch_edge_counts<float>(const Geom<float>&, const float*, const float*, const float*,
                                               const float*, int, int, double, int*, cudaStream_t);
template cudaError_t launch_edge_counts<double>(const Geom<double>&, const double*, const double*, const double*,
                                                const double*, int, int, double, int*, cudaStream_t);

}  // namespace stp
