// Constraint projections shared by the step and substep kernels (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace ffsrl {

// Positions are reached through an accessor with ld(slot) / st(slot, value):
// SmemX for a CTA's own shared memory (or a global working copy), the
// cluster accessor of xpbd_cluster.cu for positions spread over the shared
// memory of a thread-block cluster.
struct SmemX {
    float4* p;
    __device__ __forceinline__ float4 ld(int s) const { return p[s]; }
    __device__ __forceinline__ void st(int s, float4 v) const { p[s] = v; }
};
// The same positions reached by byte offset (slot x 16) instead of slot: for
// the record stream whose slot fields hold byte offsets (MeshDev::recs16).
struct SmemXB {
    unsigned char* p;
    __device__ __forceinline__ float4 ld(int off) const { return *reinterpret_cast<const float4*>(p + off); }
    __device__ __forceinline__ void st(int off, float4 v) const { *reinterpret_cast<float4*>(p + off) = v; }
};

// The hardware's reciprocal and reciprocal-square-root estimates (PTX
// rcp.approx.ftz / rsqrt.approx.ftz, flushing subnormals): the projections'
// operands are normal numbers (|x_ab|^2 is at least min_len2, denominators
// are sums of inverse masses and compliances).
__device__ __forceinline__ float rcp_est(float x) {
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ __forceinline__ float rsqrt_est(float x) {
    float y;
    asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// Edge-distance constraint C = |x_a - x_b| - d in XPBD form (Eq. 1 with
// compliance): dlambda = (-C - at lambda) / (w_a + w_b + at), x_a += w_a dlambda n,
// x_b -= w_b dlambda n, n = (x_a - x_b) / |x_a - x_b|. Applied to register
// copies; false (nothing changed) for a skipped constraint. Every rounding
// step is spelled out (fused multiply-adds where written), so all kernels
// that call this give the same bits whatever their register budget.
// LAM = false: lambda is 0 and not kept (one iteration); fma(-at, 0, -C) is
// -C exactly for a finite at >= 0, so -C is used directly (same bits).
template <bool LAM = true>
__device__ __forceinline__ bool edge_update(float4& xa, float4& xb, float d, float at, float min_len2, float& lam) {
    const float dx = __fsub_rn(xa.x, xb.x), dy = __fsub_rn(xa.y, xb.y), dz = __fsub_rn(xa.z, xb.z);
    const float l2 = __fmaf_rn(dz, dz, __fmaf_rn(dy, dy, __fmul_rn(dx, dx)));
    const float denom = __fadd_rn(__fadd_rn(xa.w, xb.w), at);
    if (l2 < min_len2 || denom == 0.f) return false;
    const float il = rsqrt_est(l2);            // 1/|x_ab| (hardware estimate)
    const float len = __fmul_rn(l2, il);
    const float C = __fsub_rn(len, d);
    const float dl = __fmul_rn(LAM ? __fmaf_rn(-at, lam, -C) : -C, rcp_est(denom));
    const float s = __fmul_rn(dl, il);
    const float sa = __fmul_rn(xa.w, s), sb = __fmul_rn(xb.w, s);
    xa.x = __fmaf_rn(sa, dx, xa.x); xa.y = __fmaf_rn(sa, dy, xa.y); xa.z = __fmaf_rn(sa, dz, xa.z);
    xb.x = __fmaf_rn(-sb, dx, xb.x); xb.y = __fmaf_rn(-sb, dy, xb.y); xb.z = __fmaf_rn(-sb, dz, xb.z);
    if (LAM) lam = __fadd_rn(lam, dl);
    return true;
}

template <bool LAM = true, class Acc>
__device__ __forceinline__ void project_edge(const Acc& X, uint2 rec, float at, float min_len2, float& lam) {
    const int a = int(rec.x & 0xffffu), b = int(rec.x >> 16);
    float4 xa = X.ld(a), xb = X.ld(b);
    if (edge_update<LAM>(xa, xb, __uint_as_float(rec.y), at, min_len2, lam)) {
        X.st(a, xa);
        X.st(b, xb);
    }
}
template <bool LAM = true>
__device__ __forceinline__ void project_edge(float4* X, uint2 rec, float at, float min_len2, float& lam) {
    project_edge<LAM>(SmemX{X}, rec, at, min_len2, lam);
}

__device__ __forceinline__ float3 sub3(float4 a, float4 b) { return make_float3(a.x - b.x, a.y - b.y, a.z - b.z); }
__device__ __forceinline__ float3 cross3(float3 a, float3 b) {
    return make_float3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ __forceinline__ float dot3(float3 a, float3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

// The same operations with their rounding spelled out.
__device__ __forceinline__ float3 sub3_rn(float4 a, float4 b) {
    return make_float3(__fsub_rn(a.x, b.x), __fsub_rn(a.y, b.y), __fsub_rn(a.z, b.z));
}
__device__ __forceinline__ float3 cross3_rn(float3 a, float3 b) {
    return make_float3(__fmaf_rn(a.y, b.z, -__fmul_rn(a.z, b.y)), __fmaf_rn(a.z, b.x, -__fmul_rn(a.x, b.z)),
                       __fmaf_rn(a.x, b.y, -__fmul_rn(a.y, b.x)));
}
__device__ __forceinline__ float dot3_rn(float3 a, float3 b) {
    return __fmaf_rn(a.z, b.z, __fmaf_rn(a.y, b.y, __fmul_rn(a.x, b.x)));
}

// Tet-volume constraint C = (x_ba x x_ca) . x_da / 6 - V0 with gradients
// g_b = x_ca x x_da / 6, g_c = x_da x x_ba / 6, g_d = x_ba x x_ca / 6,
// g_a = -(g_b + g_c + g_d) (the consistent reading of Eq. 2), scaled as in
// Eq. 3 with inverse masses and compliance: dlambda = (-C - at lambda) /
// (sum w_i |g_i|^2 + at), x_i += w_i dlambda g_i. Register copies, rounding
// spelled out as for edges; LAM as for edges.
template <bool LAM = true>
__device__ __forceinline__ bool tet_update(float4& xa, float4& xb, float4& xc, float4& xd, float V0, float at,
                                           float& lam) {
    const float3 ba = sub3_rn(xb, xa), ca = sub3_rn(xc, xa), da = sub3_rn(xd, xa);
    const float3 g1 = cross3_rn(ca, da), g2 = cross3_rn(da, ba), g3 = cross3_rn(ba, ca);  // 6 x gradient
    const float3 g0 = make_float3(-__fadd_rn(__fadd_rn(g1.x, g2.x), g3.x), -__fadd_rn(__fadd_rn(g1.y, g2.y), g3.y),
                                  -__fadd_rn(__fadd_rn(g1.z, g2.z), g3.z));
    const float C = __fmaf_rn(dot3_rn(g3, da), 1.0f / 6.0f, -V0);
    const float sw = __fmaf_rn(xd.w, dot3_rn(g3, g3),
                               __fmaf_rn(xc.w, dot3_rn(g2, g2), __fmaf_rn(xb.w, dot3_rn(g1, g1),
                                                                          __fmul_rn(xa.w, dot3_rn(g0, g0)))));
    const float denom = __fmaf_rn(sw, 1.0f / 36.0f, at);
    if (denom == 0.f) return false;
    const float dl = __fmul_rn(LAM ? __fmaf_rn(-at, lam, -C) : -C, rcp_est(denom));
    const float s = __fmul_rn(dl, 1.0f / 6.0f);
    const float sa = __fmul_rn(xa.w, s), sb = __fmul_rn(xb.w, s), sc = __fmul_rn(xc.w, s), sd = __fmul_rn(xd.w, s);
    xa.x = __fmaf_rn(sa, g0.x, xa.x); xa.y = __fmaf_rn(sa, g0.y, xa.y); xa.z = __fmaf_rn(sa, g0.z, xa.z);
    xb.x = __fmaf_rn(sb, g1.x, xb.x); xb.y = __fmaf_rn(sb, g1.y, xb.y); xb.z = __fmaf_rn(sb, g1.z, xb.z);
    xc.x = __fmaf_rn(sc, g2.x, xc.x); xc.y = __fmaf_rn(sc, g2.y, xc.y); xc.z = __fmaf_rn(sc, g2.z, xc.z);
    xd.x = __fmaf_rn(sd, g3.x, xd.x); xd.y = __fmaf_rn(sd, g3.y, xd.y); xd.z = __fmaf_rn(sd, g3.z, xd.z);
    if (LAM) lam = __fadd_rn(lam, dl);
    return true;
}

template <bool LAM = true, class Acc>
__device__ __forceinline__ void project_tet(const Acc& X, uint4 rec, float at, float& lam) {
    const int a = int(rec.x & 0xffffu), b = int(rec.x >> 16);
    const int c = int(rec.y & 0xffffu), d = int(rec.y >> 16);
    float4 xa = X.ld(a), xb = X.ld(b), xc = X.ld(c), xd = X.ld(d);
    if (tet_update<LAM>(xa, xb, xc, xd, __uint_as_float(rec.z), at, lam)) {
        X.st(a, xa);
        X.st(b, xb);
        X.st(c, xc);
        X.st(d, xd);
    }
}
template <bool LAM = true>
__device__ __forceinline__ void project_tet(float4* X, uint4 rec, float at, float& lam) {
    project_tet<LAM>(SmemX{X}, rec, at, lam);
}

// Tissue connection (Sec. III-A): C = |x_v - p| - d0 with p the centroid of
// face (a, b, c); gradients n = (x_v - p)/|x_v - p| at v and -n/3 at a, b, c,
// so sum w |g|^2 = w_v + (w_a + w_b + w_c)/9; XPBD step with the distance
// compliance. Skipped when |x_v - p|^2 < min_len2 or the denominator is 0.
// Rounding is spelled out so every build gives the same bits.
template <class Acc>
__device__ __forceinline__ void project_conn(const Acc& X, uint4 rec, float at, float min_len2, float& lam) {
    const int v = int(rec.x & 0xffffu), a = int(rec.x >> 16);
    const int b = int(rec.y & 0xffffu), c = int(rec.y >> 16);
    const float d0 = __uint_as_float(rec.z);
    float4 xv = X.ld(v), xa = X.ld(a), xb = X.ld(b), xc = X.ld(c);
    const float third = 1.0f / 3.0f;
    const float rx = __fsub_rn(xv.x, __fmul_rn(__fadd_rn(__fadd_rn(xa.x, xb.x), xc.x), third));
    const float ry = __fsub_rn(xv.y, __fmul_rn(__fadd_rn(__fadd_rn(xa.y, xb.y), xc.y), third));
    const float rz = __fsub_rn(xv.z, __fmul_rn(__fadd_rn(__fadd_rn(xa.z, xb.z), xc.z), third));
    const float l2 = __fadd_rn(__fadd_rn(__fmul_rn(rx, rx), __fmul_rn(ry, ry)), __fmul_rn(rz, rz));
    const float denom = __fadd_rn(__fadd_rn(xv.w, __fmul_rn(__fadd_rn(__fadd_rn(xa.w, xb.w), xc.w), 1.0f / 9.0f)), at);
    if (l2 < min_len2 || denom == 0.f) return;
    const float len = sqrtf(l2);
    const float C = __fsub_rn(len, d0);
    const float dl = __fdiv_rn(__fsub_rn(-C, __fmul_rn(at, lam)), denom);
    const float s = __fdiv_rn(dl, len);
    const float sv = __fmul_rn(xv.w, s);
    xv.x = __fadd_rn(xv.x, __fmul_rn(sv, rx));
    xv.y = __fadd_rn(xv.y, __fmul_rn(sv, ry));
    xv.z = __fadd_rn(xv.z, __fmul_rn(sv, rz));
    float4* f[3] = {&xa, &xb, &xc};
    for (int k = 0; k < 3; ++k) {
        const float sk = __fmul_rn(__fmul_rn(f[k]->w, s), third);
        f[k]->x = __fsub_rn(f[k]->x, __fmul_rn(sk, rx));
        f[k]->y = __fsub_rn(f[k]->y, __fmul_rn(sk, ry));
        f[k]->z = __fsub_rn(f[k]->z, __fmul_rn(sk, rz));
    }
    X.st(v, xv);
    X.st(a, xa);
    X.st(b, xb);
    X.st(c, xc);
    lam = __fadd_rn(lam, dl);
}
__device__ __forceinline__ void project_conn(float4* X, uint4 rec, float at, float min_len2, float& lam) {
    project_conn(SmemX{X}, rec, at, min_len2, lam);
}

// Jacobi forms (the paper's parallel scheme, Sec. III-A): the same steps
// evaluated at the given positions, returning the corrections instead of
// applying them (zero for a skipped constraint) and carrying lambda.
__device__ __forceinline__ void edge_delta(const float4* X, uint2 rec, float at, float min_len2, float& lam,
                                          float3& da, float3& db) {
    const int a = int(rec.x & 0xffffu), b = int(rec.x >> 16);
    const float d = __uint_as_float(rec.y);
    const float4 xa = X[a], xb = X[b];
    const float dx = xa.x - xb.x, dy = xa.y - xb.y, dz = xa.z - xb.z;
    const float l2 = dx * dx + dy * dy + dz * dz;
    const float denom = xa.w + xb.w + at;
    da = make_float3(0.f, 0.f, 0.f);
    db = da;
    if (l2 < min_len2 || denom == 0.f) return;
    const float len = sqrtf(l2);
    const float C = len - d;
    const float dl = __fdividef(-C - at * lam, denom);
    const float s = __fdividef(dl, len);
    const float sa = xa.w * s, sb = xb.w * s;
    da = make_float3(sa * dx, sa * dy, sa * dz);
    db = make_float3(-(sb * dx), -(sb * dy), -(sb * dz));
    lam += dl;
}

__device__ __forceinline__ void tet_delta(const float4* X, uint4 rec, float at, float& lam, float3* dxs) {
    const int a = int(rec.x & 0xffffu), b = int(rec.x >> 16);
    const int c = int(rec.y & 0xffffu), d = int(rec.y >> 16);
    const float V0 = __uint_as_float(rec.z);
    const float4 xa = X[a], xb = X[b], xc = X[c], xd = X[d];
    const float3 ba = sub3(xb, xa), ca = sub3(xc, xa), da = sub3(xd, xa);
    const float3 g1 = cross3(ca, da), g2 = cross3(da, ba), g3 = cross3(ba, ca);  // 6 x gradient
    const float3 g0 = make_float3(-(g1.x + g2.x + g3.x), -(g1.y + g2.y + g3.y), -(g1.z + g2.z + g3.z));
    const float C = dot3(g3, da) * (1.0f / 6.0f) - V0;
    const float sw = xa.w * dot3(g0, g0) + xb.w * dot3(g1, g1) + xc.w * dot3(g2, g2) + xd.w * dot3(g3, g3);
    const float denom = sw * (1.0f / 36.0f) + at;
    for (int i = 0; i < 4; ++i) dxs[i] = make_float3(0.f, 0.f, 0.f);
    if (denom == 0.f) return;
    const float dl = __fdividef(-C - at * lam, denom);
    const float s = dl * (1.0f / 6.0f);
    const float sa = xa.w * s, sb = xb.w * s, sc = xc.w * s, sd = xd.w * s;
    dxs[0] = make_float3(sa * g0.x, sa * g0.y, sa * g0.z);
    dxs[1] = make_float3(sb * g1.x, sb * g1.y, sb * g1.z);
    dxs[2] = make_float3(sc * g2.x, sc * g2.y, sc * g2.z);
    dxs[3] = make_float3(sd * g3.x, sd * g3.y, sd * g3.z);
    lam += dl;
}

// Largest relative violation of an edge record: |C| / d.
__device__ __forceinline__ float edge_violation(const float4* X, uint2 rec) {
    const float4 xa = X[rec.x & 0xffffu], xb = X[rec.x >> 16];
    const float dx = xa.x - xb.x, dy = xa.y - xb.y, dz = xa.z - xb.z;
    const float d = __uint_as_float(rec.y);
    return fabsf(sqrtf(dx * dx + dy * dy + dz * dz) - d) / d;
}

// Relative violation of a tet record: |C| / |V0|.
__device__ __forceinline__ float tet_violation(const float4* X, uint4 rec) {
    const float4 xa = X[rec.x & 0xffffu], xb = X[rec.x >> 16], xc = X[rec.y & 0xffffu], xd = X[rec.y >> 16];
    const float3 ba = sub3(xb, xa), ca = sub3(xc, xa), da = sub3(xd, xa);
    const float V0 = __uint_as_float(rec.z);
    return fabsf(dot3(cross3(ba, ca), da) * (1.0f / 6.0f) - V0) / fabsf(V0);
}

}  // namespace ffsrl
