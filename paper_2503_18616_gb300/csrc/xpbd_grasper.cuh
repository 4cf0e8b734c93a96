// The paper's grasper tool on the GPU (Sec. III-A "Surgical tool model" and
// "Collisions"): three capsules -- the shaft from the remote centre of motion
// to the tool point, two clamps leaving the tool point at +-alpha from the
// shaft axis in the plane of the axis and world x -- against the surface
// faces of the tissue. A face whose closest point to a capsule axis lies
// within the capsule radius is pushed out along the penetration direction by
// a PBD step of stiffness 1 on its vertices, weighted by the barycentric
// coordinates of that point. Closest points between a segment and a triangle
// are computed exactly: the segment's crossing of the triangle, else the
// nearest of each segment end against the triangle and each triangle edge
// against the segment (the Voronoi-region point-triangle test and the
// clamped segment-segment solution of Ericson, Real-Time Collision
// Detection, Sec. 5.1.5 and 5.1.9).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "xpbd_device.cuh"

namespace ffsrl {

struct Capsules {
    float a[3][3], b[3][3];   // segment ends of shaft, clamp +, clamp -
    float r[3];
    // for the faces' reach test: axis b - a, 1 / |b - a|^2 (0 for a point),
    // and the largest coordinate magnitude of a plus that of b
    float ax[3][3], inv_la2[3], qscale[3];
};

// Every product and sum below is rounded on its own (no fused multiply-add),
// so the compiler cannot fuse them differently in different kernels: the
// grasper gives the same bits under every execution schedule.
__device__ __forceinline__ float fm(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ float fa(float a, float b) { return __fadd_rn(a, b); }
__device__ __forceinline__ float fs(float a, float b) { return __fsub_rn(a, b); }
__device__ __forceinline__ float3 f3sub(float3 a, float3 b) { return make_float3(fs(a.x, b.x), fs(a.y, b.y), fs(a.z, b.z)); }
__device__ __forceinline__ float f3dot(float3 a, float3 b) { return fa(fa(fm(a.x, b.x), fm(a.y, b.y)), fm(a.z, b.z)); }
__device__ __forceinline__ float3 f3cross(float3 a, float3 b) {
    return make_float3(fs(fm(a.y, b.z), fm(a.z, b.y)), fs(fm(a.z, b.x), fm(a.x, b.z)), fs(fm(a.x, b.y), fm(a.y, b.x)));
}
__device__ __forceinline__ float3 f3axpy(float s, float3 x, float3 y) {   // y + s x
    return make_float3(fa(y.x, fm(s, x.x)), fa(y.y, fm(s, x.y)), fa(y.z, fm(s, x.z)));
}
__device__ __forceinline__ float3 f3scale(float s, float3 x) { return make_float3(fm(s, x.x), fm(s, x.y), fm(s, x.z)); }
__device__ __forceinline__ float3 f3bary(const float* w, float3 a, float3 b, float3 c) {
    return make_float3(fa(fa(fm(w[0], a.x), fm(w[1], b.x)), fm(w[2], c.x)),
                       fa(fa(fm(w[0], a.y), fm(w[1], b.y)), fm(w[2], c.y)),
                       fa(fa(fm(w[0], a.z), fm(w[1], b.z)), fm(w[2], c.z)));
}

// Unit shaft axis from the remote centre towards tool point c.
__device__ __forceinline__ float3 grasper_axis(const MeshDev& M, float3 cc) {
    const float3 rcm = make_float3(M.rcm[0], M.rcm[1], M.rcm[2]);
    const float3 d = f3sub(cc, rcm);
    const float L = sqrtf(f3dot(d, d));
    return L > 0.f ? make_float3(d.x / L, d.y / L, d.z / L) : make_float3(0.f, 0.f, -1.f);
}

// The dragging point: the end of the closed clamps, clamp_length beyond the
// tool point along the shaft axis.
__device__ __forceinline__ float3 grasper_drag_point(const SimDev& S, const MeshDev& M, const double* c) {
    const float3 cc = make_float3(float(c[0]), float(c[1]), float(c[2]));
    return f3axpy(S.clamp_length, grasper_axis(M, cc), cc);
}

// Capsules of the grasper at tool point c with clamp opening cs = (cos, sin).
__device__ __forceinline__ void grasper_capsules(const SimDev& S, const MeshDev& M, const double* c, float2 cs,
                                                 Capsules& K) {
    const float3 rcm = make_float3(M.rcm[0], M.rcm[1], M.rcm[2]);
    const float3 cc = make_float3(float(c[0]), float(c[1]), float(c[2]));
    const float3 d = grasper_axis(M, cc);
    float3 u = make_float3(fs(1.f, fm(d.x, d.x)), -fm(d.x, d.y), -fm(d.x, d.z));   // e_x minus its part along d
    if (sqrtf(f3dot(u, u)) < 1e-6f) u = make_float3(-fm(d.y, d.x), fs(1.f, fm(d.y, d.y)), -fm(d.y, d.z));
    const float lu = sqrtf(f3dot(u, u));
    u = make_float3(u.x / lu, u.y / lu, u.z / lu);
    const float lc = S.clamp_length, ca = cs.x, sa = cs.y;
    const float3 dp = f3axpy(sa, u, f3scale(ca, d)), dm = f3axpy(-sa, u, f3scale(ca, d));
    const float3 e1 = f3axpy(lc, dp, cc), e2 = f3axpy(lc, dm, cc);
    const float3 A[3] = {rcm, cc, cc}, B[3] = {cc, e1, e2};
    for (int k = 0; k < 3; ++k) {
        K.a[k][0] = A[k].x; K.a[k][1] = A[k].y; K.a[k][2] = A[k].z;
        K.b[k][0] = B[k].x; K.b[k][1] = B[k].y; K.b[k][2] = B[k].z;
    }
    K.r[0] = S.shaft_radius;
    K.r[1] = K.r[2] = S.clamp_radius;
    for (int k = 0; k < 3; ++k) {
        const float3 ax = make_float3(B[k].x - A[k].x, B[k].y - A[k].y, B[k].z - A[k].z);
        const float la2 = ax.x * ax.x + ax.y * ax.y + ax.z * ax.z;
        K.ax[k][0] = ax.x; K.ax[k][1] = ax.y; K.ax[k][2] = ax.z;
        K.inv_la2[k] = la2 > 0.f ? 1.f / la2 : 0.f;
        K.qscale[k] = fmaxf(fmaxf(fabsf(A[k].x), fabsf(A[k].y)), fabsf(A[k].z)) +
                      fmaxf(fmaxf(fabsf(B[k].x), fabsf(B[k].y)), fabsf(B[k].z));
    }
}

// Closest point of triangle (a, b, c) to x: barycentric weights w.
__device__ __forceinline__ void tri_closest(float3 x, float3 a, float3 b, float3 c, float* w) {
    const float3 ab = f3sub(b, a), ac = f3sub(c, a), ax = f3sub(x, a), bx = f3sub(x, b), cx = f3sub(x, c);
    const float d1 = f3dot(ab, ax), d2 = f3dot(ac, ax), d3 = f3dot(ab, bx), d4 = f3dot(ac, bx);
    const float d5 = f3dot(ab, cx), d6 = f3dot(ac, cx);
    const float vc = fs(fm(d1, d4), fm(d3, d2)), vb = fs(fm(d5, d2), fm(d1, d6)), va = fs(fm(d3, d6), fm(d5, d4));
    if (d1 <= 0.f && d2 <= 0.f) { w[0] = 1.f; w[1] = 0.f; w[2] = 0.f; }
    else if (d3 >= 0.f && d4 <= d3) { w[0] = 0.f; w[1] = 1.f; w[2] = 0.f; }
    else if (vc <= 0.f && d1 >= 0.f && d3 <= 0.f) { const float t = d1 / fs(d1, d3); w[0] = fs(1.f, t); w[1] = t; w[2] = 0.f; }
    else if (d6 >= 0.f && d5 <= d6) { w[0] = 0.f; w[1] = 0.f; w[2] = 1.f; }
    else if (vb <= 0.f && d2 >= 0.f && d6 <= 0.f) { const float t = d2 / fs(d2, d6); w[0] = fs(1.f, t); w[1] = 0.f; w[2] = t; }
    else if (va <= 0.f && fs(d4, d3) >= 0.f && fs(d5, d6) >= 0.f) {
        const float t = fs(d4, d3) / fa(fs(d4, d3), fs(d5, d6));
        w[0] = 0.f; w[1] = fs(1.f, t); w[2] = t;
    } else {
        const float den = fa(fa(va, vb), vc);
        w[1] = vb / den; w[2] = vc / den; w[0] = fs(fs(1.f, w[1]), w[2]);
    }
}

__device__ __forceinline__ float clamp01(float t) { return t < 0.f ? 0.f : (t > 1.f ? 1.f : t); }

// Closest points of segments p0-p1 and q0-q1: parameters s, t.
__device__ __forceinline__ void seg_closest(float3 p0, float3 p1, float3 q0, float3 q1, float& s, float& t) {
    const float3 d1 = f3sub(p1, p0), d2 = f3sub(q1, q0), r = f3sub(p0, q0);
    const float a = f3dot(d1, d1), e = f3dot(d2, d2), f = f3dot(d2, r);
    const float tiny = 1e-30f;
    if (a <= tiny && e <= tiny) { s = 0.f; t = 0.f; return; }
    if (a <= tiny) { s = 0.f; t = clamp01(f / e); return; }
    const float c = f3dot(d1, r);
    if (e <= tiny) { t = 0.f; s = clamp01(-c / a); return; }
    const float b = f3dot(d1, d2), den = fs(fm(a, e), fm(b, b));
    s = den != 0.f ? clamp01(fs(fm(b, f), fm(c, e)) / den) : 0.f;
    t = fa(fm(b, s), f) / e;
    if (t < 0.f) { t = 0.f; s = clamp01(-c / a); }
    else if (t > 1.f) { t = 1.f; s = clamp01(fs(b, c) / a); }
}

// Closest points of segment q0-q1 and triangle (a, b, c): returns the distance,
// the triangle point's barycentric weights w and the segment point q.
__device__ __forceinline__ float seg_tri_closest(float3 q0, float3 q1, float3 a, float3 b, float3 c, float* w,
                                                 float3& q) {
    const float3 ab = f3sub(b, a), ac = f3sub(c, a), n = f3cross(ab, ac), dq = f3sub(q1, q0);
    const float den = f3dot(n, dq);
    if (den != 0.f) {
        const float t = f3dot(n, f3sub(a, q0)) / den;
        if (t >= 0.f && t <= 1.f) {
            const float3 y = f3axpy(t, dq, q0);
            float wy[3];
            tri_closest(y, a, b, c, wy);
            if (wy[0] > 0.f && wy[1] > 0.f && wy[2] > 0.f) {
                w[0] = wy[0]; w[1] = wy[1]; w[2] = wy[2];
                q = y;
                return 0.f;
            }
        }
    }
    float best = -1.f;
    const float3 ends[2] = {q0, q1};
    for (int e = 0; e < 2; ++e) {
        float we[3];
        tri_closest(ends[e], a, b, c, we);
        const float3 dd = f3sub(f3bary(we, a, b, c), ends[e]);
        const float d = sqrtf(f3dot(dd, dd));
        if (best < 0.f || d < best) {
            best = d;
            w[0] = we[0]; w[1] = we[1]; w[2] = we[2];
            q = ends[e];
        }
    }
    const float3 tv[3] = {a, b, c};
    for (int e = 0; e < 3; ++e) {
        const float3 u = tv[e], v = tv[e == 2 ? 0 : e + 1];
        float s_, t_;
        seg_closest(q0, q1, u, v, s_, t_);
        const float3 cq = f3axpy(s_, dq, q0), cp = f3axpy(t_, f3sub(v, u), u);
        const float3 dd = f3sub(cp, cq);
        const float d = sqrtf(f3dot(dd, dd));
        if (d < best) {
            best = d;
            w[0] = 0.f; w[1] = 0.f; w[2] = 0.f;
            w[e] = fs(1.f, t_);
            w[e == 2 ? 0 : e + 1] = t_;
            q = cq;
        }
    }
    return best;
}

// Bounding sphere of face (a, b, c) about its centroid g, with the largest
// coordinate magnitude of g (for the reach test's margin).
struct FaceSphere {
    float3 g;
    float rho, gmax;
};
__device__ __forceinline__ FaceSphere face_sphere(float3 a, float3 b, float3 c) {
    FaceSphere F;
    F.g = make_float3((a.x + b.x + c.x) * (1.f / 3.f), (a.y + b.y + c.y) * (1.f / 3.f), (a.z + b.z + c.z) * (1.f / 3.f));
    const float3 ga = make_float3(a.x - F.g.x, a.y - F.g.y, a.z - F.g.z),
                 gb = make_float3(b.x - F.g.x, b.y - F.g.y, b.z - F.g.z),
                 gc = make_float3(c.x - F.g.x, c.y - F.g.y, c.z - F.g.z);
    F.rho = sqrtf(fmaxf(fmaxf(ga.x * ga.x + ga.y * ga.y + ga.z * ga.z, gb.x * gb.x + gb.y * gb.y + gb.z * gb.z),
                        gc.x * gc.x + gc.y * gc.y + gc.z * gc.z));
    F.gmax = fmaxf(fmaxf(fabsf(F.g.x), fabsf(F.g.y)), fabsf(F.g.z));
    return F;
}

// Whether the face lies certainly farther than r_k from capsule k's axis
// segment: the distance from the face's centroid to the segment, less the
// radius of the face's bounding sphere, is at least r_k plus a margin of
// 1e-3 r_k + 1e-5 x (the largest coordinate of g, plus those of the segment's
// ends). The second term is about a hundred times the rounding error of these
// sums and of the exact closest-point distance (a few ulp of the
// coordinates), so a face this test rejects is one the exact test below
// would leave alone: skipping it does not change any bit.
__device__ __forceinline__ bool face_out_of_reach(const FaceSphere& F, const Capsules& K, int k) {
    const float3 ax = make_float3(K.ax[k][0], K.ax[k][1], K.ax[k][2]);
    const float3 rg = make_float3(F.g.x - K.a[k][0], F.g.y - K.a[k][1], F.g.z - K.a[k][2]);
    float t = (rg.x * ax.x + rg.y * ax.y + rg.z * ax.z) * K.inv_la2[k];
    t = t < 0.f ? 0.f : (t > 1.f ? 1.f : t);
    const float3 dv = make_float3(rg.x - t * ax.x, rg.y - t * ax.y, rg.z - t * ax.z);
    const float d = sqrtf(dv.x * dv.x + dv.y * dv.y + dv.z * dv.z);
    return d - F.rho >= K.r[k] * 1.001f + 1e-5f * (F.gmax + K.qscale[k]);
}

// Pushes one surface face out of the three capsules (shaft, then clamps).
// X is the env's position array (slot order). With `bits` set (last substep)
// the free vertices a push moves are marked in the contact bits (vertex ids).
__device__ __forceinline__ void grasper_face(float4* X, uint4 rec, const Capsules& K, float tiny_len, unsigned* bits,
                                          const uint16_t* vert_of) {
    const int ia = int(rec.x & 0xffffu), ib = int(rec.x >> 16), ic = int(rec.y & 0xffffu), io = int(rec.y >> 16);
    // loaded once: only this thread moves the face's vertices while it
    // processes the face (faces of one colour share no vertex), so after a push
    // the registers hold what the next capsule would read back
    float4 xa = X[ia], xb = X[ib], xc = X[ic];
    // the face's bounding sphere, computed again after a push moves the face
    FaceSphere F = face_sphere(make_float3(xa.x, xa.y, xa.z), make_float3(xb.x, xb.y, xb.z), make_float3(xc.x, xc.y, xc.z));
    for (int k = 0; k < 3; ++k) {
        if (face_out_of_reach(F, K, k)) continue;
        const float3 a = make_float3(xa.x, xa.y, xa.z), b = make_float3(xb.x, xb.y, xb.z), c = make_float3(xc.x, xc.y, xc.z);
        const float3 q0 = make_float3(K.a[k][0], K.a[k][1], K.a[k][2]), q1 = make_float3(K.b[k][0], K.b[k][1], K.b[k][2]);
        float w[3];
        float3 q;
        const float dist = seg_tri_closest(q0, q1, a, b, c, w, q);
        if (!(dist < K.r[k])) continue;
        float3 n;
        if (dist > tiny_len) {
            const float3 pq = f3sub(f3bary(w, a, b, c), q);
            n = make_float3(pq.x / dist, pq.y / dist, pq.z / dist);
        } else {
            // the axis crosses the face: radially from the axis through the
            // centroid, or (centroid on the axis too) into the tissue
            const float3 g = make_float3(fa(fa(a.x, b.x), c.x) / 3.f, fa(fa(a.y, b.y), c.y) / 3.f,
                                         fa(fa(a.z, b.z), c.z) / 3.f);
            const float3 ax = f3sub(q1, q0), rel = f3sub(g, q0);
            const float la2 = f3dot(ax, ax);
            const float tt = la2 > 0.f ? f3dot(rel, ax) / la2 : 0.f;
            n = f3axpy(-tt, ax, rel);
            float ln = sqrtf(f3dot(n, n));
            if (!(ln > tiny_len)) {
                n = f3cross(f3sub(b, a), f3sub(c, a));
                ln = sqrtf(f3dot(n, n));
                if (!(ln > 0.f)) continue;
                const float4 xo = X[io];
                if (f3dot(n, make_float3(fs(xo.x, a.x), fs(xo.y, a.y), fs(xo.z, a.z))) < 0.f) ln = -ln;
            }
            n = make_float3(n.x / ln, n.y / ln, n.z / ln);
        }
        const float C = fs(dist, K.r[k]);
        const float den = fa(fa(fm(fm(xa.w, w[0]), w[0]), fm(fm(xb.w, w[1]), w[1])), fm(fm(xc.w, w[2]), w[2]));
        if (!(den > 0.f)) continue;
        const float sc = C / den;
        const float ga = fm(fm(xa.w, w[0]), sc), gb = fm(fm(xb.w, w[1]), sc), gc = fm(fm(xc.w, w[2]), sc);
        xa.x = fs(xa.x, fm(ga, n.x)); xa.y = fs(xa.y, fm(ga, n.y)); xa.z = fs(xa.z, fm(ga, n.z));
        xb.x = fs(xb.x, fm(gb, n.x)); xb.y = fs(xb.y, fm(gb, n.y)); xb.z = fs(xb.z, fm(gb, n.z));
        xc.x = fs(xc.x, fm(gc, n.x)); xc.y = fs(xc.y, fm(gc, n.y)); xc.z = fs(xc.z, fm(gc, n.z));
        X[ia] = xa;
        X[ib] = xb;
        X[ic] = xc;
        F = face_sphere(make_float3(xa.x, xa.y, xa.z), make_float3(xb.x, xb.y, xb.z), make_float3(xc.x, xc.y, xc.z));
        if (bits) {
            const int sl[3] = {ia, ib, ic};
            const float wv[3] = {xa.w, xb.w, xc.w};
            for (int i = 0; i < 3; ++i)
                if (wv[i] > 0.f && w[i] > 0.f) {
                    const int v = vert_of[sl[i]];
                    atomicOr(&bits[v >> 5], 1u << (v & 31));
                }
        }
    }
}

// Dragging constraint: the grasped vertex (slot sv) kept at distance d0 from
// the dragging point g, stiffness 1, the tool kinematic.
__device__ __forceinline__ void grasper_drag(float4* X, int sv, float3 g, float d0) {
    float4 x = X[sv];
    const float3 dv = make_float3(fs(x.x, g.x), fs(x.y, g.y), fs(x.z, g.z));
    const float len = sqrtf(f3dot(dv, dv));
    if (!(len > 0.f)) return;
    const float C = fs(len, d0);
    x.x = fs(x.x, fm(C, dv.x) / len);
    x.y = fs(x.y, fm(C, dv.y) / len);
    x.z = fs(x.z, fm(C, dv.z) / len);
    X[sv] = x;
}

}  // namespace ffsrl
