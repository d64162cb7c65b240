// Device geometry shared by the setup kernels and the per-frequency near fill
// of the conventional-AIM mode: 3-vectors, source-triangle frames, the
// closed-form potentials of a flat triangle, and the mesh view.

#pragma once

#include <cmath>

namespace aimx {

struct V3 {
    double x, y, z;
};
__host__ __device__ inline V3 v3(double x, double y, double z) { return V3{x, y, z}; }
__host__ __device__ inline V3 operator+(V3 a, V3 b) { return v3(a.x + b.x, a.y + b.y, a.z + b.z); }
__host__ __device__ inline V3 operator-(V3 a, V3 b) { return v3(a.x - b.x, a.y - b.y, a.z - b.z); }
__host__ __device__ inline V3 operator*(double s, V3 a) { return v3(s * a.x, s * a.y, s * a.z); }
__host__ __device__ inline double dot(V3 a, V3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__host__ __device__ inline V3 cross(V3 a, V3 b) {
    return v3(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}
__device__ inline double norm3(V3 a) { return sqrt(dot(a, a)); }
__device__ inline V3 load3(const double* p) { return v3(p[0], p[1], p[2]); }

// ------------------------------------------------------------------ static triangle potentials

// Frame of a source triangle for the closed-form potentials of 1/R.
struct TriFrame {
    V3 v[3];
    V3 n;        // unit normal (right-hand rule on v0, v1, v2)
    V3 lh[3];    // unit edge vectors v_i -> v_{i+1}
    V3 mh[3];    // outward in-plane edge normals lh x n
    double scale;
};

__device__ inline void make_frame(TriFrame& T, V3 a, V3 b, V3 c) {
    T.v[0] = a;
    T.v[1] = b;
    T.v[2] = c;
    V3 cr = cross(b - a, c - a);
    T.n = (1.0 / norm3(cr)) * cr;
    double smax = 0.0;
    for (int i = 0; i < 3; ++i) {
        V3 e = T.v[(i + 1) % 3] - T.v[i];
        double L = norm3(e);
        smax = fmax(smax, L);
        T.lh[i] = (1.0 / L) * e;
        T.mh[i] = cross(T.lh[i], T.n);
    }
    T.scale = smax;
}

// I1 = int 1/R dS', J = int (r' - rho)/R dS', G = grad_r I1, rho = projection of r.
// Edge-sum closed forms from the surface divergence theorem; the normal
// component of G uses sgn(d) = 0 on the plane (principal value).
__device__ inline void tri_potentials(const TriFrame& T, V3 r, double& I1, V3& J, V3& G, V3& rho) {
    double d = dot(r - T.v[0], T.n);
    rho = r - d * T.n;
    double ad = fabs(d);
    double sgn = (ad <= 1e-12 * T.scale) ? 0.0 : (d > 0 ? 1.0 : -1.0);
    double i1 = 0.0, bsum = 0.0;
    V3 j = v3(0, 0, 0), g = v3(0, 0, 0);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        V3 a = T.v[i], b = T.v[(i + 1) % 3];
        double sm = dot(a - rho, T.lh[i]);
        double sp = dot(b - rho, T.lh[i]);
        double t0 = dot(a - rho, T.mh[i]);
        double Rm = norm3(r - a);
        double Rp = norm3(r - b);
        double R02 = t0 * t0 + d * d;
        double f2 = (sp + sm >= 0.0) ? log((Rp + sp) / (Rm + sm)) : log((Rm - sm) / (Rp - sp));
        double beta = atan2(t0 * sp, R02 + ad * Rp) - atan2(t0 * sm, R02 + ad * Rm);
        i1 += t0 * f2;
        bsum += beta;
        j = j + (0.5 * (R02 * f2 + sp * Rp - sm * Rm)) * T.mh[i];
        g = g - f2 * T.mh[i];
    }
    I1 = i1 - ad * bsum;
    J = j;
    G = g - (sgn * bsum) * T.n;
}

// Potentials of the linear kernel R = |r - r'| (Sec. III-A-3):
//   IR = int_T R dS',   JR = int_T (rho' - rho) R dS'.
// With d the signed height of r over T and the per-edge quantities above,
//   div'((rho' - rho) R) = 3 R - d^2 / R  gives  IR = (d^2 I1 + sum_i t0 E1_i) / 3,
//   grad'(R^3) = 3 R (rho' - rho)           gives  JR = sum_i m_i E3_i / 3,
// where E1 = int_edge R dl and E3 = int_edge R^3 dl in closed form.  f2 is set
// to 0 where R0 = 0 (every term it enters carries a factor R0^2 or t0 there).
__device__ inline void tri_r_potentials(const TriFrame& T, V3 r, double& IR, V3& JR, V3& rho) {
    double d = dot(r - T.v[0], T.n);
    rho = r - d * T.n;
    double ad = fabs(d);
    double i1 = 0.0, bsum = 0.0, e1 = 0.0;
    V3 j = v3(0, 0, 0);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
        V3 a = T.v[i], b = T.v[(i + 1) % 3];
        double sm = dot(a - rho, T.lh[i]);
        double sp = dot(b - rho, T.lh[i]);
        double t0 = dot(a - rho, T.mh[i]);
        double Rm = norm3(r - a);
        double Rp = norm3(r - b);
        double R02 = t0 * t0 + d * d;
        double f2 = 0.0;
        if (R02 > 0.0) f2 = (sp + sm >= 0.0) ? log((Rp + sp) / (Rm + sm)) : log((Rm - sm) / (Rp - sp));
        double beta = atan2(t0 * sp, R02 + ad * Rp) - atan2(t0 * sm, R02 + ad * Rm);
        i1 += t0 * f2;
        bsum += beta;
        double lin = sp * Rp - sm * Rm;
        e1 += t0 * 0.5 * (lin + R02 * f2);
        double E3 = 0.25 * (sp * Rp * Rp * Rp - sm * Rm * Rm * Rm) + 0.375 * R02 * lin + 0.375 * R02 * R02 * f2;
        j = j + E3 * T.mh[i];
    }
    double I1 = i1 - ad * bsum;
    IR = (d * d * I1 + e1) / 3.0;
    JR = (1.0 / 3.0) * j;
}

// ------------------------------------------------------------------ mesh view

struct GeomView {
    const double* xyz;
    const int* tri;
    const double* area;
    const int* btri;    // [N][2]
    const int* bfree;   // [N][2]
    const double* blen; // [N]
};

__device__ inline V3 vtx(const GeomView& g, int t, int k) { return load3(g.xyz + 3 * g.tri[3 * t + k]); }

}  // namespace aimx
