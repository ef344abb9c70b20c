// Immersed-boundary kernels: MLS interpolation at markers and hydrodynamic
// probes (Sec. 2.2, Eqs. uLag, l2norm, intKernel; Sec. 2.3, Eqs. hydroForP,
// hydroForNu), membrane forces + Verlet update + spreading (Sec. 2.3,
// Eqs. strainFor, bendFor, volFor, newtonSoft, verletPos, verletVel;
// Sec. 2.2, Eq. bodyforce) and the rigid-body Newton-Euler update
// (Eqs. linearVelRig, angularVelRig).
//
// Per step and body: k_moments streams the populations once for every node
// of the body's support region (predictor density and velocity), k_mls
// fits at every marker and probe from those node moments, and one
// structure kernel updates the markers and spreads the IB force.
#include "lbib_device.cuh"
#include "lbib_kernels.h"
#include "sweep_cell.cuh"

namespace lbib {

constexpr int kPts = 32;          // MLS points per block
constexpr int kMlsThreads = 256;  // 8 warps, 4 points each
static_assert(kPts <= 32 && kPts % (kMlsThreads / 32) == 0, "one lane per point in phases 0 and 2");
constexpr double kAlpha = 0.3;    // Eq. (intKernel)
constexpr double kRw = 1.3;       // support size r_w (Sec. 2.2)
constexpr double kProbe = 1.2;    // probe length (Sec. 2.3)
constexpr int kBoxLo = 3, kBoxHi = 4;  // node margins that cover marker and probe supports

__device__ __forceinline__ float rcp(float x) { return __frcp_rn(x); }
__device__ __forceinline__ double rcp(double x) { return 1.0 / x; }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// ---------------------------------------------------------------------------
// Predictor moments on the support region: for every node of the box,
// pull the 19 populations (f_i(x) = f*_i(x - e_i)) and store
// rho - 1 and u* = (sum f e + g_ext/2)/rho.  Grid-stride over the box
// recorded on the device by the previous step's update.
// ---------------------------------------------------------------------------
// Support-region moments, node-interleaved: mom[4 node + q] holds rho - 1
// and the predictor velocity u*_x, u*_y, u*_z of node `node`, so that the
// MLS gather of one support node is a single 16-byte (FP32) or two
// 16-byte (FP64) loads.
__device__ __forceinline__ void mom_store(float *m, int node, float a, float b, float c, float d) {
    reinterpret_cast<float4 *>(m)[node] = make_float4(a, b, c, d);
}
__device__ __forceinline__ void mom_store(double *m, int node, double a, double b, double c, double d) {
    reinterpret_cast<double2 *>(m)[2 * node] = make_double2(a, b);
    reinterpret_cast<double2 *>(m)[2 * node + 1] = make_double2(c, d);
}
template <bool kCG>
__device__ __forceinline__ void mom_load(const float *m, int node, float *v) {
    const float4 q = ld_ro<kCG>(reinterpret_cast<const float4 *>(m) + node);
    v[0] = q.x;
    v[1] = q.y;
    v[2] = q.z;
    v[3] = q.w;
}
template <bool kCG>
__device__ __forceinline__ void mom_load(const double *m, int node, double *v) {
    const double2 a = ld_ro<kCG>(reinterpret_cast<const double2 *>(m) + 2 * node);
    const double2 b = ld_ro<kCG>(reinterpret_cast<const double2 *>(m) + 2 * node + 1);
    v[0] = a.x;
    v[1] = a.y;
    v[2] = b.x;
    v[3] = b.y;
}

template <typename S, typename R, bool kCG = false>
__device__ __forceinline__ void moments_body(const S *__restrict__ fin, const Lattice &L, const int *__restrict__ box,
                                             int *__restrict__ box_next, R *__restrict__ mom,
                                             uint32_t *__restrict__ step_inc, const int vb, const int nvb) {
    // the step counter and the support box are read and written by other
    // kernels of the step (or other work items of a persistent launch):
    // L2 accesses, coherent across SMs
    if (step_inc && vb == 0 && threadIdx.x == 0) atomicAdd(step_inc, 1u);  // read by the later kernels of the step
    const int n[3] = {L.nx, L.ny, L.nz};
    int lo[3], ext[3];
    for (int a = 0; a < 3; ++a) {
        long long l = __ldcg(box + a), h = __ldcg(box + 3 + a);
        if (L.bc[a] == kWall) {
            l = l < 0 ? 0 : l;
            h = h > n[a] - 1 ? n[a] - 1 : h;
        } else if (h - l + 1 > n[a]) {
            l = 0;
            h = n[a] - 1;
        }
        lo[a] = (int)l;
        ext[a] = h < l ? 0 : (int)(h - l + 1);
    }
    if (vb == 0 && threadIdx.x < 6) box_next[threadIdx.x] = threadIdx.x < 3 ? 0x7fffffff : (int)0x80000000;
    const int total = ext[0] * ext[1] * ext[2];
    const int nxy = L.nx * L.ny;
    const long long st = L.stride;
    for (int k = vb * blockDim.x + threadIdx.x; k < total; k += nvb * blockDim.x) {
        int c[3] = {lo[0] + k % ext[0], lo[1] + (k / ext[0]) % ext[1], lo[2] + k / (ext[0] * ext[1])};
        int cm[3], cp[3];
        for (int a = 0; a < 3; ++a) {
            if (L.bc[a] == kPeriodic) c[a] = wrap_periodic(c[a], n[a]);
            int vm = c[a] - 1, vp = c[a] + 1;
            if (vm < 0) vm = L.bc[a] == kPeriodic ? n[a] - 1 : 0;
            if (vp >= n[a]) vp = L.bc[a] == kPeriodic ? 0 : n[a] - 1;
            cm[a] = vm;
            cp[a] = vp;
        }
        R drho = R(0), jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int sx = ex(i) > 0 ? cm[0] : ex(i) < 0 ? cp[0] : c[0];
            const int sy = ey(i) > 0 ? cm[1] : ey(i) < 0 ? cp[1] : c[1];
            const int sz = ez(i) > 0 ? cm[2] : ez(i) < 0 ? cp[2] : c[2];
            const R gi = Pop<S, R>::from(ld_ro<kCG>(fin + (long long)i * st + (sx + L.nx * sy + nxy * sz)));
            drho += gi;
            if (ex(i) > 0) jx += gi;
            if (ex(i) < 0) jx -= gi;
            if (ey(i) > 0) jy += gi;
            if (ey(i) < 0) jy -= gi;
            if (ez(i) > 0) jz += gi;
            if (ez(i) < 0) jz -= gi;
        }
        const int node = c[0] + L.nx * c[1] + nxy * c[2];
        const R rho = R(1) + drho;
        mom_store(mom, node, drho, (jx + R(0.5) * pick<R>(L.gext_d[0], L.gext_f[0])) / rho,
                  (jy + R(0.5) * pick<R>(L.gext_d[1], L.gext_f[1])) / rho,
                  (jz + R(0.5) * pick<R>(L.gext_d[2], L.gext_f[2])) / rho);
    }
}

template <typename S, typename R>
__global__ void __launch_bounds__(256) k_moments(const S *__restrict__ fin, Lattice L, const int *__restrict__ box,
                                                 int *__restrict__ box_next, R *__restrict__ mom,
                                                 uint32_t *__restrict__ step_inc) {
    chain_release();  // the MLS kernel may be scheduled beside this one
    moments_body<S, R>(fin, L, box, box_next, mom, step_inc, blockIdx.x, gridDim.x);
}

constexpr int kSums = 26;  // A (10 entries), b for rho (4), b for u (12)

// Shared memory of the MLS phases.  The per-point sums are formed through a
// shared-memory transpose (red) in the MLS kernels, which run alone and are
// fastest that way, or with kShfl by warp shuffles (the persistent batched
// step, whose shared memory is taken from the L1 its sweep items need).
template <typename R, bool kShfl = false>
struct MlsSmem {
    // per point, filled in phase 0 (one lane per point)
    double frac[kPts][3];  // X - base, exact
    int base[kPts][3];
    R fracR[kPts][3];
    R nrm[kPts][3];
    double vol[kPts];
    // per point and support node, kept for the transfer weights of markers
    // (with kShfl the offsets x_k - X are formed again from fracR instead)
    R W[kPts][27];
    R d[kShfl ? 1 : kPts][27][3];
    // per point: A = sum W p p^T, b_f = sum W p (f - f_c) for f = rho - 1, u_x, u_y, u_z
    R sums[kPts][kSums];
    R ref[kPts][4];   // the fitted fields at the support's centre node (the fits are of f - ref)
    R row0[kPts][4];  // first row of A^-1
    int pid[kPts];    // point of each slot (-1 past the end): slots follow the body's cell order
    // per warp: transpose buffer of the 26 products of each node (unused with kShfl)
    R red[kShfl ? 1 : kMlsThreads / 32][kSums][kShfl ? 1 : 33];
};

// Sums 32 values per lane over the warp (a reduce-scatter butterfly): at
// offset h each lane keeps the half of its values whose index bit h it
// holds and receives the partner's partial sums of that half, so that lane
// q ends with the total of value q (31 shuffles, no shared memory).
template <typename R>
__device__ __forceinline__ R warp_reduce_scatter32(R (&v)[32], const int lane) {
#pragma unroll
    for (int h = 16; h >= 1; h >>= 1) {
        const bool up = (lane & h) != 0;
#pragma unroll
        for (int i = 0; i < h; ++i) {
            const R send = up ? v[i] : v[i + h];
            const R keep = up ? v[i + h] : v[i];
            v[i] = keep + __shfl_xor_sync(0xffffffffu, send, h);
        }
    }
    return v[0];
}

// 1/d in FP64 from the FP32 reciprocal refined by two Newton steps
// (relative error ~1e-7 -> ~1e-14 -> below the double rounding).  d must lie
// in the FP32 normal range, or the seed is infinite or zero: callers bound it.
__device__ __forceinline__ double recip64(double d) {
    double r = (double)__frcp_rn((float)d);
    r = fma(r, fma(-d, r, 1.0), r);
    r = fma(r, fma(-d, r, 1.0), r);
    return r;
}

// Inverse of a symmetric positive definite 4x4 matrix given by its upper
// triangle (00,01,02,03,11,12,13,22,23,33), as the adjugate over the
// determinant, both from the 2x2 minors of the top and bottom row pairs
// (a shallow dependency chain: FP64 latency, not throughput, limits this
// per-point solve).  Returns false unless kMinDet < determinant < kMaxDet:
// the bounds keep the FP32 seed of recip64 finite and normal.  An MLS moment
// matrix has entries of at most 27 * 1.5^2 (weights <= 1, offsets <= 1.5),
// so det < 4e7 always, and the centre node with the three nearer face
// neighbours (all within 1.22 of the point: weights >= 5e-5, unit offsets)
// keep det above ~1e-16; a determinant outside the bounds marks a singular
// support.
constexpr double kMinDet = 1e-30, kMaxDet = 1e30;
__device__ bool spd_inverse4(const double *a, double *inv) {
    const double m00 = a[0], m01 = a[1], m02 = a[2], m03 = a[3];
    const double m11 = a[4], m12 = a[5], m13 = a[6], m22 = a[7], m23 = a[8], m33 = a[9];
    // rows 0,1 and rows 2,3 (symmetric: m10 = m01, ...)
    const double s0 = m00 * m11 - m01 * m01;
    const double s1 = m00 * m12 - m02 * m01;
    const double s2 = m00 * m13 - m03 * m01;
    const double s3 = m01 * m12 - m02 * m11;
    const double s4 = m01 * m13 - m03 * m11;
    const double s5 = m02 * m13 - m03 * m12;
    const double c5 = m22 * m33 - m23 * m23;
    const double c4 = m12 * m33 - m13 * m23;
    const double c3 = m12 * m23 - m13 * m22;
    const double c2 = m02 * m33 - m03 * m23;
    const double c1 = m02 * m23 - m03 * m22;
    const double c0 = m02 * m13 - m03 * m12;
    const double det = s0 * c5 - s1 * c4 + s2 * c3 + s3 * c2 - s4 * c1 + s5 * c0;
    if (!(det > kMinDet && det < kMaxDet)) return false;
    const double id = recip64(det);
    // rows of the adjugate (the matrix is symmetric, so is its inverse)
    inv[0] = (m11 * c5 - m12 * c4 + m13 * c3) * id;
    inv[1] = (-m01 * c5 + m02 * c4 - m03 * c3) * id;
    inv[2] = (m13 * s5 - m23 * s4 + m33 * s3) * id;
    inv[3] = (-m12 * s5 + m22 * s4 - m23 * s3) * id;
    inv[5] = (m00 * c5 - m02 * c2 + m03 * c1) * id;
    inv[6] = (-m03 * s5 + m23 * s2 - m33 * s1) * id;
    inv[7] = (m02 * s5 - m22 * s2 + m23 * s1) * id;
    inv[10] = (m03 * s4 - m13 * s2 + m33 * s0) * id;
    inv[11] = (-m02 * s4 + m12 * s2 - m23 * s0) * id;
    inv[15] = (m02 * s3 - m12 * s1 + m22 * s0) * id;
    inv[4] = inv[1];
    inv[8] = inv[2];
    inv[9] = inv[6];
    inv[12] = inv[3];
    inv[13] = inv[7];
    inv[14] = inv[11];
    return true;
}

// Inverse of a symmetric positive definite 4x4 matrix (upper triangle as for
// spd_inverse4) in FP32, by Cholesky: A = L L^T, M = L^-1 by forward
// substitution, A^-1 = M^T M.  Backward stable, so for moment sums that are
// themselves FP32 it is as accurate as an FP64 inverse of the same sums
// (both leave errors of the order of the sums' own rounding in the fits),
// at FP32 issue rates.  Returns false unless every pivot is positive and
// finite (a singular support).
__device__ bool spd_inverse4_chol(const float *a, float *inv) {
    const float d0 = a[0];
    if (!(d0 > 0.f && d0 < 1e30f)) return false;
    const float l00 = sqrtf(d0), r0 = 1.f / l00;
    const float l10 = a[1] * r0, l20 = a[2] * r0, l30 = a[3] * r0;
    const float d1 = a[4] - l10 * l10;
    if (!(d1 > 0.f)) return false;
    const float l11 = sqrtf(d1), r1 = 1.f / l11;
    const float l21 = (a[5] - l20 * l10) * r1, l31 = (a[6] - l30 * l10) * r1;
    const float d2 = a[7] - l20 * l20 - l21 * l21;
    if (!(d2 > 0.f)) return false;
    const float l22 = sqrtf(d2), r2 = 1.f / l22;
    const float l32 = (a[8] - l30 * l20 - l31 * l21) * r2;
    const float d3 = a[9] - l30 * l30 - l31 * l31 - l32 * l32;
    if (!(d3 > 0.f)) return false;
    const float r3 = 1.f / sqrtf(d3);
    // M = L^-1 (lower triangular)
    const float m00 = r0;
    const float m10 = -l10 * m00 * r1, m11 = r1;
    const float m20 = -(l20 * m00 + l21 * m10) * r2, m21 = -l21 * m11 * r2, m22 = r2;
    const float m30 = -(l30 * m00 + l31 * m10 + l32 * m20) * r3, m31 = -(l31 * m11 + l32 * m21) * r3,
                m32 = -l32 * m22 * r3, m33 = r3;
    // (M^T M)_ij = sum_{k >= max(i, j)} m_ki m_kj
    inv[0] = m00 * m00 + m10 * m10 + m20 * m20 + m30 * m30;
    inv[1] = m10 * m11 + m20 * m21 + m30 * m31;
    inv[2] = m20 * m22 + m30 * m32;
    inv[3] = m30 * m33;
    inv[5] = m11 * m11 + m21 * m21 + m31 * m31;
    inv[6] = m21 * m22 + m31 * m32;
    inv[7] = m31 * m33;
    inv[10] = m22 * m22 + m32 * m32;
    inv[11] = m32 * m33;
    inv[15] = m33 * m33;
    inv[4] = inv[1];
    inv[8] = inv[2];
    inv[9] = inv[6];
    inv[12] = inv[3];
    inv[13] = inv[7];
    inv[14] = inv[11];
    return true;
}

// Squared distance with the products and sums rounded one by one in the
// order (x^2 + y^2) + z^2, as a plain sum of squares is.
__device__ __forceinline__ double dist2_exact(double a, double b, double c) {
    return __dadd_rn(__dadd_rn(__dmul_rn(a, a), __dmul_rn(b, b)), __dmul_rn(c, c));
}

// MLS at markers and probes, 32 points per block.  Points 0..nm-1 are the
// markers (the vertices, or the triangle centroids); point nm + 2t + side is
// the probe of triangle t on the outer (side 0) or inner (side 1) face.  With p_k = (1, x_k - X) the fit of a
// field f is a = A^-1 b_f, A = sum_k W_k p_k p_k^T, b_f = sum_k W_k p_k f_k
// (Eq. l2norm), i.e. f(X) = a_0 and grad f = (a_1, a_2, a_3).
//  phase 0: one lane per point: position (probes: triangle geometry), the
//           nearest node base = floor(X + 1/2) and the exact offset X - base;
//  phase 1: one warp per point, one lane per support node: weight
//           W = exp(-(r/alpha)^2) for r <= 1 (the cut-off decided exactly as
//           in FP64), node moments less those of the centre node f_c, the
//           26 products W p p^T and W p (f - f_c), summed over the nodes;
//  phase 2: one lane per point: inverse of A (FP64 adjugate in the FP64
//           path, FP32 Cholesky in the FP32 one); markers get
//           U = (A^-1 b_u)_0 + u_c (Eq. uLag), probes the pressure c_s^2 rho and
//           the traction rho nu (grad u + grad u^T) . n from the fits;
//  phase 3: markers keep phi_k = W_k (A^-1 p_k)_0 for spreading.
template <typename R, bool kCG = false, bool kShfl = false>
__device__ __forceinline__ void mls_body(const R *__restrict__ mom, const Lattice &L, const BodyView &B, int *err,
                                         MlsSmem<R, kShfl> &sm, const int vb, const int nvb) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nm = B.nm, npts = nm + 2 * B.nt;
    const int p0 = vb * kPts;
    const int nxy = L.nx * L.ny;
    const int n[3] = {L.nx, L.ny, L.nz};

    // The lane-per-point phases (0 and 2) run FP64 code; FP64 issues per
    // warp-instruction on one SM sub-partition, so blocks rotate the warp
    // that runs them over the four sub-partitions.
    const int w0 = vb & 3, w2 = (vb + 2) & 3;

    // ---------------- phase 0: one lane per point ----------------
    if (warp == w0 && lane < kPts) {
        const int slot = p0 + lane;
        const int p = slot < npts ? (B.perm ? B.perm[slot] : slot) : -1;
        sm.pid[lane] = p;
        sm.vol[lane] = 0.0;
        if (p >= 0) {
            double P[3];
            if (p < nm && B.centroid) {
                const int *tv = B.tri + 3 * p;
                for (int a = 0; a < 3; ++a) P[a] = (B.X[3 * tv[0] + a] + B.X[3 * tv[1] + a] + B.X[3 * tv[2] + a]) / 3.0;
            } else if (p < nm) {
                P[0] = B.X[3 * p];
                P[1] = B.X[3 * p + 1];
                P[2] = B.X[3 * p + 2];
            } else {
                // probe X_c +- 1.2 n, with X_c = x_0 + (e1 + e2)/3 and the
                // triangle's edges and normal from origin-relative positions
                const int t = (p - nm) >> 1, side = (p - nm) & 1;
                const int *tv = B.tri + 3 * t;
                const R *Xr = (const R *)B.Xrel;
                R r0[3], e1[3], e2[3];
                for (int a = 0; a < 3; ++a) {
                    r0[a] = Xr[3 * tv[0] + a];
                    e1[a] = Xr[3 * tv[1] + a] - r0[a];
                    e2[a] = Xr[3 * tv[2] + a] - r0[a];
                }
                const R N[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2],
                                e1[0] * e2[1] - e1[1] * e2[0]};
                const R nn = sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
                const R inn = R(1) / nn, sg = side ? R(-kProbe) : R(kProbe);
                for (int a = 0; a < 3; ++a) {
                    const R nr = N[a] * inn, c3 = (e1[a] + e2[a]) / R(3);
                    sm.nrm[lane][a] = nr;
                    P[a] = B.X[3 * tv[0] + a] + (double)(c3 + sg * nr);
                    if (side == 0) {
                        R *tg = (R *)B.tri_geo + 8 * t;
                        tg[a] = nr;
                        tg[4 + a] = r0[a] + c3;
                    }
                }
                if (side == 0) {
                    ((R *)B.tri_geo)[8 * t + 3] = R(0.5) * nn;
                    const double v6 = (double)r0[0] * (double)N[0] + (double)r0[1] * (double)N[1] +
                                      (double)r0[2] * (double)N[2];
                    B.tri_vol[t] = v6;
                    sm.vol[lane] = v6;
                }
            }
            bool bad = false, diverged = false;
            for (int a = 0; a < 3; ++a) {
                if (!(fabs(P[a]) < kMaxMarkerCoord)) {  // non-finite or runaway: flag, keep indices sane
                    diverged = true;
                    P[a] = 0.0;
                }
                int b = __double2int_rd(P[a] + 0.5);  // floor(X + 1/2)
                if (L.bc[a] == kWall && (b - 1 < 1 || b + 1 > n[a] - 2)) {
                    bad = true;
                    b = b < 2 ? 2 : (b > n[a] - 3 ? n[a] - 3 : b);
                }
                sm.base[lane][a] = b;
                sm.frac[lane][a] = P[a] - (double)b;
                sm.fracR[lane][a] = R(sm.frac[lane][a]);
            }
            if (diverged)
                atomicCAS(err, 0, kErrDiverged);
            else if (bad)
                atomicCAS(err, 0, kErrBodyWall);
        }
    }
    __syncthreads();

    // ---------------- phase 1: one warp per point, one lane per node ----------------
    // The gathers of the warp's points are issued together, then each
    // point's weights and products are reduced in turn.
    constexpr int kPerWarp = kPts / (kMlsThreads / 32);
    R gu[kPerWarp][4];
#pragma unroll
    for (int j = 0; j < kPerWarp; ++j) {
        const int lp = warp * kPerWarp + j;
        const int p = sm.pid[lp];
        gu[j][0] = gu[j][1] = gu[j][2] = gu[j][3] = R(0);
        if (p >= 0 && lane < 27) {
            const int dd[3] = {lane % 3 - 1, (lane / 3) % 3 - 1, lane / 9 - 1};
            int cw[3];
            for (int a = 0; a < 3; ++a) {
                int cc = sm.base[lp][a] + dd[a];
                if (L.bc[a] == kPeriodic) {
                    if (cc < 0)
                        cc += n[a];
                    else if (cc >= n[a])
                        cc -= n[a];
                    if (cc < 0 || cc >= n[a]) cc = ((cc % n[a]) + n[a]) % n[a];
                }
                cw[a] = cc;
            }
            const int node = cw[0] + L.nx * cw[1] + nxy * cw[2];
            mom_load<kCG>(mom, node, gu[j]);
            if (p < nm) {
                gu[j][0] = R(0);  // markers use the velocity fit only
                B.node[27 * p + lane] = node;
            }
        }
    }
#pragma unroll
    for (int j = 0; j < kPerWarp; ++j) {
        const int lp = warp * kPerWarp + j;
        const int p = sm.pid[lp];
        if (p < 0) break;
        // fit f - f_c, f_c the moments of the centre node (lane 13, always in
        // the support): the same fit, since MLS reproduces constants, but
        // the sums and the solve then carry the field's variation over the
        // support rather than its size, which the gradients at the probes
        // (small differences of the fitted values) need
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            const R fc = __shfl_sync(0xffffffffu, gu[j][c], 13);
            gu[j][c] -= fc;
            if (lane == 0) sm.ref[lp][c] = fc;
        }
        R W = R(0), dk[3] = {R(0), R(0), R(0)};
        if (lane < 27) {
            const int dd[3] = {lane % 3 - 1, (lane / 3) % 3 - 1, lane / 9 - 1};
            // x_k - X = dd - (X - base), one rounding like (base + dd) - X
            for (int a = 0; a < 3; ++a) dk[a] = R(dd[a]) - sm.fracR[lp][a];
            // support cut-off r_k <= 1 of Eq. (intKernel), decided on the FP64
            // squared distance; the FP32 path computes it in FP64 only near
            // the cut-off, where its own rounding could flip the decision
            bool inside;
            R dist2;
            if (sizeof(R) == 8) {
                dist2 = R(dist2_exact(double(dk[0]), double(dk[1]), double(dk[2])));
                inside = double(dist2) <= L.dist2_cut;
            } else {
                dist2 = dk[0] * dk[0] + dk[1] * dk[1] + dk[2] * dk[2];
                if (fabsf(float(dist2) - L.dist2_cut_f) > 1e-4f) {
                    inside = float(dist2) < L.dist2_cut_f;
                } else {
                    const double e0 = (double)dd[0] - sm.frac[lp][0], e1 = (double)dd[1] - sm.frac[lp][1],
                                 e2 = (double)dd[2] - sm.frac[lp][2];
                    inside = dist2_exact(e0, e1, e2) <= L.dist2_cut;
                }
            }
            if (inside) {
                const R r = sqrt(dist2) / R(kRw);
                W = exp(-(r / R(kAlpha)) * (r / R(kAlpha)));
            }
            sm.W[lp][lane] = W;
            if constexpr (!kShfl)
                for (int a = 0; a < 3; ++a) sm.d[lp][lane][a] = dk[a];
        }
        // the 26 products of this node (zero on lanes 27..31), summed over
        // the support nodes: lane q forms sum q
        const R Wd[4] = {W, W * dk[0], W * dk[1], W * dk[2]};
        if constexpr (kShfl) {
            R v[32];
            v[0] = Wd[0];
            v[1] = Wd[1];
            v[2] = Wd[2];
            v[3] = Wd[3];
            v[4] = Wd[1] * dk[0];
            v[5] = Wd[1] * dk[1];
            v[6] = Wd[1] * dk[2];
            v[7] = Wd[2] * dk[1];
            v[8] = Wd[2] * dk[2];
            v[9] = Wd[3] * dk[2];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                v[10 + q] = Wd[q] * gu[j][0];
                v[14 + q] = Wd[q] * gu[j][1];
                v[18 + q] = Wd[q] * gu[j][2];
                v[22 + q] = Wd[q] * gu[j][3];
            }
#pragma unroll
            for (int q = kSums; q < 32; ++q) v[q] = R(0);
            const R sum = warp_reduce_scatter32(v, lane);
            if (lane < kSums) sm.sums[lp][lane] = sum;
        } else {
            R(*red)[33] = sm.red[warp];
            red[0][lane] = Wd[0];
            red[1][lane] = Wd[1];
            red[2][lane] = Wd[2];
            red[3][lane] = Wd[3];
            red[4][lane] = Wd[1] * dk[0];
            red[5][lane] = Wd[1] * dk[1];
            red[6][lane] = Wd[1] * dk[2];
            red[7][lane] = Wd[2] * dk[1];
            red[8][lane] = Wd[2] * dk[2];
            red[9][lane] = Wd[3] * dk[2];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                red[10 + q][lane] = Wd[q] * gu[j][0];
                red[14 + q][lane] = Wd[q] * gu[j][1];
                red[18 + q][lane] = Wd[q] * gu[j][2];
                red[22 + q][lane] = Wd[q] * gu[j][3];
            }
            __syncwarp();
            if (lane < kSums) {
                R acc = R(0);
#pragma unroll
                for (int k = 0; k < 27; ++k) acc += red[lane][k];
                sm.sums[lp][lane] = acc;
            }
            __syncwarp();
        }
    }
    __syncthreads();

    // ---------------- phase 2: one lane per point ----------------
    if (warp == w2 && lane < kPts && sm.pid[lane] >= 0) {
        const int p = sm.pid[lane];
        const R *S = sm.sums[lane];
        R Ai[16];
        if constexpr (sizeof(R) == 8) {
            double a[10], inv[16];
            for (int q = 0; q < 10; ++q) a[q] = (double)S[q];
            if (!spd_inverse4(a, inv)) atomicCAS(err, 0, -1);
            for (int q = 0; q < 16; ++q) Ai[q] = R(inv[q]);
        } else {
            float a[10];
            for (int q = 0; q < 10; ++q) a[q] = (float)S[q];
            if (!spd_inverse4_chol(a, (float *)Ai)) atomicCAS(err, 0, -1);
        }
        const R *fc = sm.ref[lane];
        if (p < nm) {
            for (int q = 0; q < 4; ++q) sm.row0[lane][q] = Ai[q];
            double *Uo = B.centroid ? B.Uc : B.U;
            for (int jj = 0; jj < 3; ++jj) {
                const R *bu = S + 14 + 4 * jj;
                Uo[3 * p + jj] = (double)(Ai[0] * bu[0] + Ai[1] * bu[1] + Ai[2] * bu[2] + Ai[3] * bu[3] + fc[1 + jj]);
            }
        } else {
            // fits: c_f[i] = sum_m Ai[i][m] b_f[m], plus the centre value for
            // the value (i = 0)
            R cr[4], cu[3][4];
            for (int i = 0; i < 4; ++i) {
                cr[i] = Ai[4 * i] * S[10] + Ai[4 * i + 1] * S[11] + Ai[4 * i + 2] * S[12] + Ai[4 * i + 3] * S[13];
                for (int jj = 0; jj < 3; ++jj) {
                    const R *bu = S + 14 + 4 * jj;
                    cu[jj][i] = Ai[4 * i] * bu[0] + Ai[4 * i + 1] * bu[1] + Ai[4 * i + 2] * bu[2] + Ai[4 * i + 3] * bu[3];
                }
            }
            cr[0] += fc[0];
            for (int jj = 0; jj < 3; ++jj) cu[jj][0] += fc[1 + jj];
            const int t = (p - nm) >> 1, side = (p - nm) & 1;
            const R rho = R(1) + cr[0];
            const R nu = pick<R>(L.nu_d, L.nu_f);
            R *pr = (R *)B.probe + 8 * t + 4 * side;
            pr[0] = cr[0] / R(3);  // p - c_s^2 rho0
            for (int jj = 0; jj < 3; ++jj) {
                R acc = R(0);
                for (int m = 0; m < 3; ++m) acc += rho * nu * (cu[jj][1 + m] + cu[m][1 + jj]) * sm.nrm[lane][m];
                pr[1 + jj] = acc;
            }
        }
    }
    // enclosed volume (membranes): fixed-order partial per block; the last
    // block to finish sums the partials with a fixed-shape tree
    // (deterministic whichever block is last)
    __shared__ int s_last;
    if (!B.rigid) {
        if (threadIdx.x == 32 * ((w2 + 1) & 3)) {
            double s = 0.0;
            for (int k = 0; k < kPts; ++k) s += sm.vol[k];
            B.vol_part[vb] = s;
            __threadfence();
            s_last = atomicAdd(B.vol_count, 1u) == (unsigned)nvb - 1;
        }
        __syncthreads();
        if (s_last) {
            __threadfence();
            double s = 0.0;
            for (int k = threadIdx.x; k < nvb; k += blockDim.x) s += __ldcg(B.vol_part + k);
            s = warp_sum(s);
            __shared__ double wpart[kMlsThreads / 32];
            if (lane == 0) wpart[warp] = s;
            __syncthreads();
            if (threadIdx.x == 0) {
                double tot = 0.0;
                for (int w = 0; w < kMlsThreads / 32; ++w) tot += wpart[w];
                *B.vol_sum = tot;
                *B.vol_count = 0u;
            }
        }
    }
    __syncthreads();

    // ---------------- phase 3: transfer weights of the markers ----------------
    for (int j = 0; j < kPerWarp; ++j) {
        const int lp = warp * kPerWarp + j;
        const int p = sm.pid[lp];
        if (p < 0) break;
        if (p >= nm) continue;  // probes keep no transfer weights
        if (lane < 27) {
            R dk[3];
            if constexpr (kShfl) {
                const int dd[3] = {lane % 3 - 1, (lane / 3) % 3 - 1, lane / 9 - 1};
                for (int a = 0; a < 3; ++a) dk[a] = R(dd[a]) - sm.fracR[lp][a];  // as in phase 1
            } else {
                for (int a = 0; a < 3; ++a) dk[a] = sm.d[lp][lane][a];
            }
            const R *r0 = sm.row0[lp];
            const R phi = sm.W[lp][lane] * (r0[0] + r0[1] * dk[0] + r0[2] * dk[1] + r0[3] * dk[2]);
            ((R *)B.phi)[27 * p + lane] = phi;
        }
    }
}

// The blocks take the nvb groups of 32 points in turn (gridDim.x = nvb
// unless the launch caps the grid).
template <typename R>
__global__ void __launch_bounds__(kMlsThreads) k_mls(const R *__restrict__ mom, Lattice L, BodyView B,
                                                     int *err, int nvb) {
    chain_wait();  // launched programmatically after the moments kernel
    extern __shared__ __align__(16) unsigned char smem_raw[];
    for (int vb = blockIdx.x; vb < nvb; vb += gridDim.x) {
        mls_body<R>(mom, L, B, err, *reinterpret_cast<MlsSmem<R> *>(smem_raw), vb, nvb);
        __syncthreads();  // the next group reuses the shared memory
    }
}

// Hydrodynamic force on triangle t from its two probes (Eqs. hydroForP,
// hydroForNu): F = [-(p+ - p-) n + (tau+ - tau-) . n] A.
template <typename R>
__device__ __forceinline__ void tri_hydro(const BodyView &B, int t, R *F) {
    const R *tg = (const R *)B.tri_geo + 8 * t;
    const R *pp = (const R *)B.probe + 8 * t, *pm = pp + 4;
    const R A = tg[3];
    for (int a = 0; a < 3; ++a) F[a] = (-(pp[0] - pm[0]) * tg[a] + (pp[1 + a] - pm[1 + a])) * A;
}

// Lanes 0..26 of a warp add c phi_k F to the force field at the support
// nodes of marker v; the lanes of the 8 block corners flag their tiles.
template <typename R>
__device__ __forceinline__ void spread_warp(const Lattice &L, const BodyView &B, int v, int lane, R c, const R *Fl,
                                            R *__restrict__ force, uint32_t *stamp, uint32_t step) {
    if (lane >= 27) return;
    const long long st = L.stride;
    const int node = B.node[27 * v + lane];
    const R w = c * ((const R *)B.phi)[27 * v + lane];
    atomicAdd(force + node, w * Fl[0]);
    atomicAdd(force + st + node, w * Fl[1]);
    atomicAdd(force + 2 * st + node, w * Fl[2]);
    if (lane == 0 || lane == 2 || lane == 6 || lane == 8 || lane == 18 || lane == 20 || lane == 24 || lane == 26) {
        const int x = node % L.nx, yz = node / L.nx, y = yz % L.ny, z = yz / L.ny;
        stamp[(x >> 3) + L.ntx * ((y >> 3) + L.nty * (z >> 3))] = step;
    }
}

// Lane k < 27 of a marker's warp adds w F to the force field at its
// support node; the lanes of the 8 block corners flag their tiles.
template <typename R>
__device__ __forceinline__ void spread_node(const Lattice &L, int lane, int node, R w, const R *Fl,
                                            R *__restrict__ force, uint32_t *stamp, uint32_t step) {
    if (lane >= 27) return;
    const long long st = L.stride;
    atomicAdd(force + node, w * Fl[0]);
    atomicAdd(force + st + node, w * Fl[1]);
    atomicAdd(force + 2 * st + node, w * Fl[2]);
    if (lane == 0 || lane == 2 || lane == 6 || lane == 8 || lane == 18 || lane == 20 || lane == 24 || lane == 26) {
        const int x = node % L.nx, yz = node / L.nx, y = yz % L.ny, z = yz / L.ny;
        stamp[(x >> 3) + L.ntx * ((y >> 3) + L.nty * (z >> 3))] = step;
    }
}

// Node box of level n+1: each block reduces its markers' cells in shared
// memory and then updates the global box once (contention on the six
// global words stays at one update per block).
struct BlockBox {
    int v[6];
    __device__ void init() {
        if (threadIdx.x < 6) v[threadIdx.x] = threadIdx.x < 3 ? 0x7fffffff : (int)0x80000000;
    }
    __device__ void add(int a, double x) {
        const int c = (int)floor(x);
        atomicMin(&v[a], c - kBoxLo);
        atomicMax(&v[3 + a], c + kBoxHi);
    }
    __device__ void flush(int *box) {
        if (threadIdx.x < 3)
            atomicMin(box + threadIdx.x, v[threadIdx.x]);
        else if (threadIdx.x < 6)
            atomicMax(box + threadIdx.x, v[threadIdx.x]);
    }
};

// Membrane vertex update, one warp per vertex: spring (Eq. strainFor),
// bending (gradient of k_b[1 - cos(theta - theta0)], reading of Eq. bendFor),
// volume penalty (restoring reading of Eq. volFor) and element hydrodynamic
// forces shared 1/3 per vertex (Eq. newtonSoft), with the lanes sharing the
// incident hinges and triangles; Verlet positions (Eqs. verletPos,
// verletVel) in FP64, one lane per component; boundary velocity
// U_b = U + F/m_v dt; the Lagrangian force F_l = U_b - U spread with
// c_l = A_l (Eq. bodyforce).
template <typename R>
__device__ __forceinline__ void membrane_body(const Lattice &L, const BodyView &B, R *__restrict__ force,
                                              uint32_t *__restrict__ stamp, const uint32_t *__restrict__ dstep,
                                              const int vb) {
    const uint32_t step = __ldcg(dstep);  // written by the moments kernel of the step
    __shared__ R s_cv;
    __shared__ BlockBox sbox;
    __shared__ R s_F[8][4];   // per vertex warp: total force (3) and vertex area
    __shared__ R s_Fl[8][3];  // per vertex warp: Lagrangian force
    __shared__ double s_U[8][3];  // centroid markers: the vertex velocity
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int v0 = vb * (blockDim.x >> 5);  // first vertex of the block
    const int v = v0 + warp;
    // the spreading lanes fetch their node and weight first
    int snode = 0;
    R sphi = R(0);
    if (!B.centroid && v < B.nv && lane < 27) {
        snode = B.node[27 * v + lane];
        sphi = ((const R *)B.phi)[27 * v + lane];
    }
    if (threadIdx.x == 0) s_cv = R(B.kv * (1.0 - *B.vol_sum * B.inv_6V0));
    sbox.init();
    __syncthreads();
    const R cv = s_cv;
    if (v < B.nv) {
    const R *Xr = (const R *)B.Xrel;
    R F[3] = {R(0), R(0), R(0)};
    for (int q = B.vh_ptr[v] + lane; q < B.vh_ptr[v + 1]; q += 32) {
        const int role = B.vh_list[q] & 3;
        const int4 H = B.vh_verts[q];
        const R *par = (const R *)B.vh_par + 4 * q;  // k_s, l0, k_b, theta0
        const R ksh = par[0], l0h = par[1], kbh = par[2], th0h = par[3];
        R e[3], ac[3], ad[3];
        for (int a = 0; a < 3; ++a) {
            const R xa = Xr[3 * H.x + a];
            e[a] = Xr[3 * H.y + a] - xa;
            ac[a] = Xr[3 * H.z + a] - xa;
            ad[a] = Xr[3 * H.w + a] - xa;
        }
        if constexpr (sizeof(R) == 4) {
            // the FP32 coordinates carry an absolute error of half an ulp of
            // the body's size; their residuals restore the edges' own relative
            // precision, which the spring extensions l - l0 and the dihedral
            // angles (small differences of the edges) need
            const float *Xl = B.Xlo;
            for (int a = 0; a < 3; ++a) {
                const float la = Xl[3 * H.x + a];
                e[a] += Xl[3 * H.y + a] - la;
                ac[a] += Xl[3 * H.z + a] - la;
                ad[a] += Xl[3 * H.w + a] - la;
            }
        }
        const R le2 = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
        const R le = sqrt(le2), ile = rcp(le);
        if (role < 2) {
            // F_a = -k (l - l0) (x_a - x_b)/l = k (l - l0) e / l, F_b = -F_a
            const R c = ksh * (le - l0h) * ile;
            const R sg = role == 0 ? R(1) : R(-1);
            for (int a = 0; a < 3; ++a) F[a] += sg * c * e[a];
        }
        const R N1[3] = {e[1] * ac[2] - e[2] * ac[1], e[2] * ac[0] - e[0] * ac[2], e[0] * ac[1] - e[1] * ac[0]};
        const R N2[3] = {ad[1] * e[2] - ad[2] * e[1], ad[2] * e[0] - ad[0] * e[2], ad[0] * e[1] - ad[1] * e[0]};
        const R l1s = N1[0] * N1[0] + N1[1] * N1[1] + N1[2] * N1[2];
        const R l2s = N2[0] * N2[0] + N2[1] * N2[1] + N2[2] * N2[2];
        const R il1 = rcp(sqrt(l1s)), il2 = rcp(sqrt(l2s));
        R n1[3], n2[3];
        for (int a = 0; a < 3; ++a) {
            n1[a] = N1[a] * il1;
            n2[a] = N2[a] * il2;
        }
        const R cx[3] = {n1[1] * n2[2] - n1[2] * n2[1], n1[2] * n2[0] - n1[0] * n2[2], n1[0] * n2[1] - n1[1] * n2[0]};
        const R theta = atan2((cx[0] * e[0] + cx[1] * e[1] + cx[2] * e[2]) * ile,
                              n1[0] * n2[0] + n1[1] * n2[1] + n1[2] * n2[2]);
        const R dth = theta - th0h;
        const R dE = B.bend_variant ? kbh * dth : kbh * sin(dth);
        const R ile2 = ile * ile;
        const R tc = (ac[0] * e[0] + ac[1] * e[1] + ac[2] * e[2]) * ile2;
        const R td = (ad[0] * e[0] + ad[1] * e[1] + ad[2] * e[2]) * ile2;
        R c1, c2;  // dtheta/dx = c1 n1/h1 + c2 n2/h2, h = |N|/|e|
        if (role == 0) {
            c1 = R(1) - tc;
            c2 = R(1) - td;
        } else if (role == 1) {
            c1 = tc;
            c2 = td;
        } else if (role == 2) {
            c1 = R(-1);
            c2 = R(0);
        } else {
            c1 = R(0);
            c2 = R(-1);
        }
        const R g1 = c1 * le * il1, g2 = c2 * le * il2;  // c / h
        for (int a = 0; a < 3; ++a) F[a] -= dE * (g1 * n1[a] + g2 * n2[a]);
    }
    // element terms: volume penalty and hydrodynamic force, 1/3 per vertex
    R Al = R(0);
    double Uv[3] = {0.0, 0.0, 0.0};
    for (int q = B.vt_ptr[v] + lane; q < B.vt_ptr[v + 1]; q += 32) {
        const int t = B.vt_list[q] / 3;
        const R *tg = (const R *)B.tri_geo + 8 * t;
        Al += tg[3] / R(3);
        R Fh[3] = {R(0), R(0), R(0)};
        if (!B.kinematic) tri_hydro<R>(B, t, Fh);  // kinematic IB: the fluid's stresses stay in the fluid
        for (int a = 0; a < 3; ++a) F[a] += (cv * tg[a] * tg[3] + Fh[a]) / R(3);
        if (B.centroid)
            for (int a = 0; a < 3; ++a) Uv[a] += (double)(tg[3] / R(3)) * B.Uc[3 * t + a];
    }
    for (int a = 0; a < 3; ++a) F[a] = warp_sum(F[a]);
    Al = warp_sum(Al);
    if (lane == 0) {
        s_F[warp][0] = F[0];
        s_F[warp][1] = F[1];
        s_F[warp][2] = F[2];
        s_F[warp][3] = Al;
    }
    if (B.centroid) {
        // the vertex moves with the area-weighted mean of its triangles'
        // centroid velocities
        for (int a = 0; a < 3; ++a) Uv[a] = warp_sum(Uv[a]);
        if (lane == 0)
            for (int a = 0; a < 3; ++a) s_U[warp][a] = Uv[a] / (double)Al;
    }
    }
    __syncthreads();
    // Newton (Eq. newtonSoft) and Verlet (Eqs. verletPos, verletVel), dt = 1,
    // in FP64 for the block's 8 vertices at once: lane 3 j + a of one warp
    // integrates component a of vertex j (FP64 issues per warp-instruction;
    // the warp rotates over the SM sub-partitions from block to block)
    if (warp == (vb & 7) && lane < 24 && v0 + lane / 3 < B.nv) {
        const int j = lane / 3, a = lane % 3, vj = v0 + j;
        const double acc = (double)s_F[j][a] * B.inv_mv;
        double U;
        if (B.centroid) {
            U = s_U[j][a];
            B.U[3 * vj + a] = U;
        } else {
            U = B.U[3 * vj + a];
        }
        const double Ub = U + acc;
        const double Fla = Ub - U;
        const double x = B.X[3 * vj + a], xp = B.Xprev[3 * vj + a];
        double xn;
        if (B.kinematic) {
            xn = x + U;  // kinematic IB: advected with the interpolated fluid velocity
        } else {
            const double xt = x + U + 0.5 * acc;
            const double ubdf = 1.5 * xt - 2.0 * x + 0.5 * xp;
            xn = x + ubdf + 0.5 * acc;
        }
        // a vertex moving a lattice unit or more in one step (or a NaN) has
        // diverged
        if (!(fabs(xn - x) < kMaxMarkerStep)) atomicCAS(B.err, 0, kErrDiverged);
        B.Xnew[3 * vj + a] = xn;
        const double rel = xn - B.origin[a];
        ((R *)B.Xrel_next)[3 * vj + a] = R(rel);
        if constexpr (sizeof(R) == 4) B.Xlo_next[3 * vj + a] = float(rel - double(float(rel)));
        B.Ub[3 * vj + a] = Ub;
        B.Fl[3 * vj + a] = Fla;
        sbox.add(a, xn);
        s_Fl[j][a] = R(Fla);
    }
    __syncthreads();
    if (!B.centroid && v < B.nv)
        spread_node<R>(L, lane, snode, s_F[warp][3] * sphi, s_Fl[warp], force, stamp, step);
    __syncthreads();
    sbox.flush(B.bbox_next);
}

template <typename R>
__global__ void __launch_bounds__(256) k_membrane(Lattice L, BodyView B, R *__restrict__ force,
                                                  uint32_t *__restrict__ stamp, const uint32_t *__restrict__ dstep,
                                                  int nvb) {
    for (int vb = blockIdx.x; vb < nvb; vb += gridDim.x) {
        membrane_body<R>(L, B, force, stamp, dstep, vb);
        __syncthreads();  // the next group of vertices reuses the shared memory
    }
}

// Rigid body: total force and moment of the element stresses, gravity
// minus buoyancy, F = m du/dt and M = I dw/dt with I in the world frame,
// second-order backward velocities (Eqs. linearVelRig, angularVelRig),
// centre and orientation advanced with the new velocities.
// One thread per triangle sums force and moment (fixed-shape block
// reduction, FP64 partial per block); the last block to finish reduces the
// partials in block order and integrates with lanes 0..8 of one warp
// working on the components side by side (FP64 issues per
// warp-instruction, so the update is written across lanes).
template <typename R>
__device__ __forceinline__ void rigid_forces_body(const BodyView &B, const int vb, const int nvb) {
    __shared__ double red[6][8];
    __shared__ int s_last;
    __shared__ double sF[6], sR[9], sY[3], sQ[4];
    double *S = B.rstate;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const R xc[3] = {R(S[RigidState::XC] - B.origin[0]), R(S[RigidState::XC + 1] - B.origin[1]),
                     R(S[RigidState::XC + 2] - B.origin[2])};
    R f[6] = {R(0), R(0), R(0), R(0), R(0), R(0)};
    const int t = vb * blockDim.x + threadIdx.x;
    if (t < B.nt && !B.rigid_force) {
        R Fh[3];
        tri_hydro<R>(B, t, Fh);
        const R *tg = (const R *)B.tri_geo + 8 * t;
        const R r[3] = {tg[4] - xc[0], tg[5] - xc[1], tg[6] - xc[2]};
        f[0] = Fh[0];
        f[1] = Fh[1];
        f[2] = Fh[2];
        f[3] = r[1] * Fh[2] - r[2] * Fh[1];
        f[4] = r[2] * Fh[0] - r[0] * Fh[2];
        f[5] = r[0] * Fh[1] - r[1] * Fh[0];
    } else if (t < B.nt && B.centroid) {
        // momentum exchange, centroid markers: minus the previous step's IB
        // force of the triangle's marker times its area, about x_c
        const R *tg = (const R *)B.tri_geo + 8 * t;
        const R c = -tg[3];
        const R Fv[3] = {c * R(B.Flc[3 * t]), c * R(B.Flc[3 * t + 1]), c * R(B.Flc[3 * t + 2])};
        const R r[3] = {tg[4] - xc[0], tg[5] - xc[1], tg[6] - xc[2]};
        f[0] = Fv[0];
        f[1] = Fv[1];
        f[2] = Fv[2];
        f[3] = r[1] * Fv[2] - r[2] * Fv[1];
        f[4] = r[2] * Fv[0] - r[0] * Fv[2];
        f[5] = r[0] * Fv[1] - r[1] * Fv[0];
    } else if (t < B.nt) {
        // momentum exchange: minus the IB force of the previous step, each
        // corner carrying a third of the triangle's area (sum_l A_l F_l)
        const R *tg = (const R *)B.tri_geo + 8 * t;
        const R c = -tg[3] / R(3);
        const R *Xr = (const R *)B.Xrel;
        for (int q = 0; q < 3; ++q) {
            const int v = B.tri[3 * t + q];
            const R Fv[3] = {c * R(B.Fl[3 * v]), c * R(B.Fl[3 * v + 1]), c * R(B.Fl[3 * v + 2])};
            const R r[3] = {Xr[3 * v] - xc[0], Xr[3 * v + 1] - xc[1], Xr[3 * v + 2] - xc[2]};
            f[0] += Fv[0];
            f[1] += Fv[1];
            f[2] += Fv[2];
            f[3] += r[1] * Fv[2] - r[2] * Fv[1];
            f[4] += r[2] * Fv[0] - r[0] * Fv[2];
            f[5] += r[0] * Fv[1] - r[1] * Fv[0];
        }
    }
    for (int q = 0; q < 6; ++q) {
        const R w = warp_sum(f[q]);
        if (lane == 0) red[q][warp] = (double)w;
    }
    __syncthreads();
    if (threadIdx.x < 6) {
        double acc = 0.0;
        for (int w = 0; w < 8; ++w) acc += red[threadIdx.x][w];
        B.vol_part[6 * vb + threadIdx.x] = acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(B.vol_count, 1u) == (unsigned)nvb - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    // totals: warp q < 6 sums partial q over the blocks, lane l taking blocks
    // l, l + 32, ... and the warp's fixed butterfly adding the lanes
    // (deterministic whichever block is last)
    if (warp < 6) {
        double acc = 0.0;
        for (int b = lane; b < nvb; b += 32) acc += __ldcg(B.vol_part + 6 * b + warp);
        acc = warp_sum(acc);
        if (lane == 0) {
            if (warp < 3) acc += (S[RigidState::DENS] - 1.0) * S[RigidState::VOL] * S[RigidState::GRAV + warp];
            // momentum exchange: the fluid inside moves with the body, rho_f V du/dt
            if (warp < 3 && B.rigid_force)
                acc += S[RigidState::VOL] * (S[RigidState::U + warp] - S[RigidState::UP + warp]);
            sF[warp] = acc;
        }
    }
    __syncthreads();
    if (warp != 0) return;
    if (lane == 0) *B.vol_count = 0u;
    __syncwarp();
    const double *q = S + RigidState::Q4;
    // rotation matrix of q, entry lane < 9
    if (lane < 9) {
        const double w = q[0], x = q[1], y = q[2], z = q[3];
        const int i = lane / 3, j = lane % 3;
        double v;
        if (i == j) {
            const double a2 = i == 0 ? y * y + z * z : i == 1 ? x * x + z * z : x * x + y * y;
            v = 1.0 - 2.0 * a2;
        } else {
            // off-diagonal 2 (u_i u_j -+ w u_k), k the third axis
            const double ui = i == 0 ? x : i == 1 ? y : z, uj = j == 0 ? x : j == 1 ? y : z;
            const int k = 3 - i - j;
            const double uk = k == 0 ? x : k == 1 ? y : z;
            const bool plus = (i == 0 && j == 2) || (i == 1 && j == 0) || (i == 2 && j == 1);
            v = 2.0 * (ui * uj + (plus ? w * uk : -w * uk));
        }
        sR[lane] = v;
    }
    __syncwarp();
    // dw/dt = I_world^-1 M = R I_b^-1 R^T M, lanes 0..2
    if (B.rigid_force) {
        // and I_f dw/dt = R I_b R^T (w - wp) rho_f / rho_s
        if (lane < 3) {
            const double *w = S + RigidState::W, *wp = S + RigidState::WP;
            sY[lane] = sR[lane] * (w[0] - wp[0]) + sR[3 + lane] * (w[1] - wp[1]) + sR[6 + lane] * (w[2] - wp[2]);
        }
        __syncwarp();
        double iy = 0.0;
        if (lane < 3) {
            const double *Ib = S + RigidState::IB + 3 * lane;
            iy = Ib[0] * sY[0] + Ib[1] * sY[1] + Ib[2] * sY[2];
        }
        __syncwarp();
        if (lane < 3) sY[lane] = iy;
        __syncwarp();
        if (lane < 3)
            sF[3 + lane] += (sR[3 * lane] * sY[0] + sR[3 * lane + 1] * sY[1] + sR[3 * lane + 2] * sY[2]) /
                            S[RigidState::DENS];
        __syncwarp();
    }
    if (lane < 3) sY[lane] = sR[lane] * sF[3] + sR[3 + lane] * sF[4] + sR[6 + lane] * sF[5];  // R^T M
    __syncwarp();
    double zl = 0.0;
    if (lane < 3) {
        const double *Ii = S + RigidState::IBINV + 3 * lane;
        zl = Ii[0] * sY[0] + Ii[1] * sY[1] + Ii[2] * sY[2];
    }
    __syncwarp();
    if (lane < 3) sY[lane] = zl;
    __syncwarp();
    // lanes 0..2: linear velocity and centre; lanes 3..5: angular velocity
    double vn = 0.0;
    if (lane < 6) {
        const int a = lane % 3;
        double vdot, v1, v2;
        if (lane < 3) {
            vdot = sF[a] * S[RigidState::INVM];
            v1 = S[RigidState::U + a];
            v2 = S[RigidState::UP + a];
        } else {
            vdot = sR[3 * a] * sY[0] + sR[3 * a + 1] * sY[1] + sR[3 * a + 2] * sY[2];
            v1 = S[RigidState::W + a];
            v2 = S[RigidState::WP + a];
        }
        vn = 2.0 / 3.0 * (2.0 * v1 - 0.5 * v2 + vdot);
    }
    __syncwarp();
    if (lane < 3) {
        const double x0 = S[RigidState::XC + lane];
        S[RigidState::XC_OLD + lane] = x0;
        S[RigidState::XC + lane] = x0 + vn;
        S[RigidState::UP + lane] = S[RigidState::U + lane];
        S[RigidState::U + lane] = vn;
    } else if (lane < 6) {
        S[RigidState::WP + lane - 3] = S[RigidState::W + lane - 3];
        S[RigidState::W + lane - 3] = vn;
    }
    // rotation by |w| about w: dq = (cos(|w|/2), sin(|w|/2) w/|w|)
    const double w0 = __shfl_sync(0xffffffffu, vn, 3), w1 = __shfl_sync(0xffffffffu, vn, 4),
                 w2 = __shfl_sync(0xffffffffu, vn, 5);
    const double th2 = w0 * w0 + w1 * w1 + w2 * w2;
    double c, sth;  // cos(|w|/2) and sin(|w|/2)/|w|
    if (th2 < 1e-6) {
        // series in x^2 = |w|^2/4 (terms beyond x^8 are below double rounding)
        const double x2 = 0.25 * th2;
        c = 1.0 + x2 * (-0.5 + x2 * (1.0 / 24.0 + x2 * (-1.0 / 720.0 + x2 * (1.0 / 40320.0))));
        sth = 0.5 * (1.0 + x2 * (-1.0 / 6.0 + x2 * (1.0 / 120.0 + x2 * (-1.0 / 5040.0))));
    } else {
        const double wl = sqrt(th2);
        double sn;
        sincos(0.5 * wl, &sn, &c);
        sth = sn / wl;
    }
    const double dq[4] = {c, sth * w0, sth * w1, sth * w2};
    double qn = q[0];
    if (th2 > 0.0 && lane < 4) {
        // component lane of dq (x) q
        if (lane == 0) qn = dq[0] * q[0] - dq[1] * q[1] - dq[2] * q[2] - dq[3] * q[3];
        if (lane == 1) qn = dq[0] * q[1] + dq[1] * q[0] + dq[2] * q[3] - dq[3] * q[2];
        if (lane == 2) qn = dq[0] * q[2] - dq[1] * q[3] + dq[2] * q[0] + dq[3] * q[1];
        if (lane == 3) qn = dq[0] * q[3] + dq[1] * q[2] - dq[2] * q[1] + dq[3] * q[0];
    } else if (lane < 4) {
        qn = q[lane];
    }
    double qq = lane < 4 ? qn * qn : 0.0;
    qq += __shfl_xor_sync(0xffffffffu, qq, 1);
    qq += __shfl_xor_sync(0xffffffffu, qq, 2);
    if (lane < 4) {
        double r = (double)rsqrtf((float)qq);  // 1/sqrt(qq), refined twice
        r = r * (1.5 - 0.5 * qq * r * r);
        r = r * (1.5 - 0.5 * qq * r * r);
        if (th2 > 0.0) qn *= r;
        sQ[lane] = qn;
        S[RigidState::Q4 + lane] = qn;
    }
    __syncwarp();
    if (lane < 9) {
        const double w = sQ[0], x = sQ[1], y = sQ[2], z = sQ[3];
        const int i = lane / 3, j = lane % 3;
        double v;
        if (i == j) {
            const double a2 = i == 0 ? y * y + z * z : i == 1 ? x * x + z * z : x * x + y * y;
            v = 1.0 - 2.0 * a2;
        } else {
            const double ui = i == 0 ? x : i == 1 ? y : z, uj = j == 0 ? x : j == 1 ? y : z;
            const int k = 3 - i - j;
            const double uk = k == 0 ? x : k == 1 ? y : z;
            const bool plus = (i == 0 && j == 2) || (i == 1 && j == 0) || (i == 2 && j == 1);
            v = 2.0 * (ui * uj + (plus ? w * uk : -w * uk));
        }
        S[RigidState::ROT + lane] = v;
    }
}

template <typename R>
__global__ void __launch_bounds__(256) k_rigid_forces(BodyView B) {
    rigid_forces_body<R>(B, blockIdx.x, gridDim.x);
}

// Rigid markers, one warp each: boundary velocity u + w x (X - x_c) of
// level n, IB force and spreading, then the markers of level n+1.
template <typename R>
__device__ __forceinline__ void rigid_markers_body(const Lattice &L, const BodyView &B, R *__restrict__ force,
                                                   uint32_t *__restrict__ stamp,
                                                   const uint32_t *__restrict__ dstep, const int vb) {
    const uint32_t step = __ldcg(dstep);  // written by the moments kernel of the step
    __shared__ BlockBox sbox;
    __shared__ R s_Al[8];
    __shared__ R s_Fl[8][3];
    __shared__ double s_U[8][3];  // centroid markers: the vertex velocity
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int v0 = vb * (blockDim.x >> 5);
    const int v = v0 + warp;
    sbox.init();
    if (v < B.nv) {
        R Al = R(0);
        double Uv[3] = {0.0, 0.0, 0.0};
        for (int q = B.vt_ptr[v] + lane; q < B.vt_ptr[v + 1]; q += 32) {
            const int t = B.vt_list[q] / 3;
            const R At3 = ((const R *)B.tri_geo)[8 * t + 3] / R(3);
            Al += At3;
            if (B.centroid)
                for (int a = 0; a < 3; ++a) Uv[a] += (double)At3 * B.Uc[3 * t + a];
        }
        Al = warp_sum(Al);
        if (lane == 0) s_Al[warp] = Al;
        if (B.centroid) {
            // the vertex velocity: area-weighted mean of its triangles'
            // centroid velocities
            for (int a = 0; a < 3; ++a) Uv[a] = warp_sum(Uv[a]);
            if (lane == 0)
                for (int a = 0; a < 3; ++a) s_U[warp][a] = Uv[a] / (double)Al;
        }
    }
    __syncthreads();
    // FP64 for the block's 8 markers at once: lane 3 j + a of one warp
    // handles component a of marker j
    if (warp == (vb & 7) && lane < 24 && v0 + lane / 3 < B.nv) {
        const int j = lane / 3, a = lane % 3, vj = v0 + j, a1 = (a + 1) % 3, a2 = (a + 2) % 3;
        const double *S = B.rstate;
        const double *un = S + RigidState::U, *wn = S + RigidState::W, *xo = S + RigidState::XC_OLD;
        const double *xc = S + RigidState::XC, *Rn = S + RigidState::ROT;
        const double r1 = B.X[3 * vj + a1] - xo[a1], r2 = B.X[3 * vj + a2] - xo[a2];
        const double ub = un[a] + (wn[a1] * r2 - wn[a2] * r1);  // (w x r)_a
        double U;
        if (B.centroid) {
            U = s_U[j][a];
            B.U[3 * vj + a] = U;
        } else {
            U = B.U[3 * vj + a];
        }
        const double Fla = ub - U;
        B.Ub[3 * vj + a] = ub;
        B.Fl[3 * vj + a] = Fla;
        const double *xb = B.Xbody + 3 * vj;
        const double xn = xc[a] + Rn[3 * a] * xb[0] + Rn[3 * a + 1] * xb[1] + Rn[3 * a + 2] * xb[2];
        // a marker moving a lattice unit or more in one step (or a NaN) has
        // diverged
        if (!(fabs(xn - B.X[3 * vj + a]) < kMaxMarkerStep)) atomicCAS(B.err, 0, kErrDiverged);
        B.Xnew[3 * vj + a] = xn;
        ((R *)B.Xrel_next)[3 * vj + a] = R(xn - B.origin[a]);
        sbox.add(a, xn);
        s_Fl[j][a] = R(Fla);
    }
    __syncthreads();
    if (!B.centroid && v < B.nv) spread_warp<R>(L, B, v, lane, s_Al[warp], s_Fl[warp], force, stamp, step);
    __syncthreads();
    sbox.flush(B.bbox_next);
}

template <typename R>
__global__ void __launch_bounds__(256) k_rigid_markers(Lattice L, BodyView B, R *__restrict__ force,
                                                       uint32_t *__restrict__ stamp, const uint32_t *__restrict__ dstep,
                                                       int nvb) {
    for (int vb = blockIdx.x; vb < nvb; vb += gridDim.x) {
        rigid_markers_body<R>(L, B, force, stamp, dstep, vb);
        __syncthreads();  // the next group of markers reuses the shared memory
    }
}

// IB force of centroid markers, one warp per triangle: the boundary
// velocity at the centroid (rigid: u + w x (X_c - x_c) of level n;
// membrane: the interpolated velocity advanced by the mean Newton
// acceleration of the triangle's vertices, which the structure kernel left
// as their Lagrangian force), F_l = U_b - U spread with c_l = A_t.
template <typename R>
__device__ __forceinline__ void centroid_body(const Lattice &L, const BodyView &B, R *__restrict__ force,
                                              uint32_t *__restrict__ stamp, const uint32_t *__restrict__ dstep,
                                              const int vb) {
    const uint32_t step = __ldcg(dstep);  // written by the moments kernel of the step
    __shared__ R s_A[8];
    __shared__ R s_Fl[8][3];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int t0 = vb * 8, t = t0 + warp;
    int snode = 0;
    R sphi = R(0);
    if (t < B.nt && lane < 27) {
        snode = B.node[27 * t + lane];
        sphi = ((const R *)B.phi)[27 * t + lane];
    }
    if (t < B.nt && lane == 0) s_A[warp] = ((const R *)B.tri_geo)[8 * t + 3];
    // FP64 for the block's 8 markers at once: lane 3 j + a of one warp
    // handles component a of marker j
    if (warp == (vb & 7) && lane < 24 && t0 + lane / 3 < B.nt) {
        const int j = lane / 3, a = lane % 3, tj = t0 + j;
        const int *tv = B.tri + 3 * tj;
        const double uc = B.Uc[3 * tj + a];
        double ub;
        if (B.rigid) {
            const int a1 = (a + 1) % 3, a2 = (a + 2) % 3;
            const double *S = B.rstate;
            const double *un = S + RigidState::U, *wn = S + RigidState::W, *xo = S + RigidState::XC_OLD;
            const double r1 = (B.X[3 * tv[0] + a1] + B.X[3 * tv[1] + a1] + B.X[3 * tv[2] + a1]) / 3.0 - xo[a1];
            const double r2 = (B.X[3 * tv[0] + a2] + B.X[3 * tv[1] + a2] + B.X[3 * tv[2] + a2]) / 3.0 - xo[a2];
            ub = un[a] + (wn[a1] * r2 - wn[a2] * r1);
        } else {
            const double acc = B.Fl[3 * tv[0] + a] + B.Fl[3 * tv[1] + a] + B.Fl[3 * tv[2] + a];
            ub = uc + acc / 3.0;
        }
        const double Fla = ub - uc;
        B.Flc[3 * tj + a] = Fla;
        s_Fl[j][a] = R(Fla);
    }
    __syncthreads();
    if (t < B.nt) spread_node<R>(L, lane, snode, s_A[warp] * sphi, s_Fl[warp], force, stamp, step);
}

template <typename R>
__global__ void __launch_bounds__(256) k_centroid_spread(Lattice L, BodyView B, R *__restrict__ force,
                                                         uint32_t *__restrict__ stamp,
                                                         const uint32_t *__restrict__ dstep) {
    centroid_body<R>(L, B, force, stamp, dstep, blockIdx.x);
}

// ---- batch kernels: the bodies of all lattices of a batch per launch ----
template <typename S, typename R>
__global__ void __launch_bounds__(256) kb_moments(BatchTables T, int phase) {
    __shared__ Lattice L;
    const int j = __ldg(T.mom_blk + blockIdx.x);
    const int vb = blockIdx.x - __ldg(T.mom_pre + j), nvb = __ldg(T.mom_pre + j + 1) - __ldg(T.mom_pre + j);
    const BodyRef &br = T.body[phase * T.nb + j];
    stage_shared(L, T.lat + br.lat);
    const LatRef &F = T.ref[phase * T.nl + br.lat];
    moments_body<S, R>((const S *)F.fin, L, br.v.bbox, br.v.bbox_next, (R *)F.mom, br.inc_step ? F.d_step : nullptr,
                       vb, nvb);
}

template <typename R>
__global__ void __launch_bounds__(kMlsThreads) kb_mls(BatchTables T, int phase) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Lattice L;
    __shared__ BodyRef br;
    const int j = __ldg(T.mls_blk + blockIdx.x);
    const int vb = blockIdx.x - __ldg(T.mls_pre + j), nvb = __ldg(T.mls_pre + j + 1) - __ldg(T.mls_pre + j);
    stage_shared(br, T.body + phase * T.nb + j);
    stage_shared(L, T.lat + br.lat);
    const LatRef &F = T.ref[phase * T.nl + br.lat];
    mls_body<R>((const R *)F.mom, L, br.v, F.err, *reinterpret_cast<MlsSmem<R> *>(smem_raw), vb, nvb);
}

template <typename R>
__global__ void __launch_bounds__(256) kb_membrane(BatchTables T, int phase) {
    __shared__ Lattice L;
    __shared__ BodyRef br;
    const int m = __ldg(T.memb_blk + blockIdx.x);
    stage_shared(br, T.body + phase * T.nb + __ldg(T.memb_id + m));
    stage_shared(L, T.lat + br.lat);
    const LatRef &F = T.ref[phase * T.nl + br.lat];
    membrane_body<R>(L, br.v, (R *)F.force, F.stamp, F.d_step, blockIdx.x - __ldg(T.memb_pre + m));
}

template <typename R>
__global__ void __launch_bounds__(256) kb_rigid_forces(BatchTables T, int phase) {
    const int m = __ldg(T.rf_blk + blockIdx.x);
    const BodyRef &br = T.body[phase * T.nb + __ldg(T.rigid_id + m)];
    const int b0 = __ldg(T.rf_pre + m);
    rigid_forces_body<R>(br.v, blockIdx.x - b0, __ldg(T.rf_pre + m + 1) - b0);
}

template <typename R>
__global__ void __launch_bounds__(256) kb_rigid_markers(BatchTables T, int phase) {
    __shared__ Lattice L;
    __shared__ BodyRef br;
    const int m = __ldg(T.rm_blk + blockIdx.x);
    stage_shared(br, T.body + phase * T.nb + __ldg(T.rigid_id + m));
    stage_shared(L, T.lat + br.lat);
    const LatRef &F = T.ref[phase * T.nl + br.lat];
    rigid_markers_body<R>(L, br.v, (R *)F.force, F.stamp, F.d_step, blockIdx.x - __ldg(T.rm_pre + m));
}

template <typename R>
__global__ void __launch_bounds__(256) kb_centroid_spread(BatchTables T, int phase) {
    __shared__ Lattice L;
    __shared__ BodyRef br;
    const int m = __ldg(T.cen_blk + blockIdx.x);
    stage_shared(br, T.body + phase * T.nb + __ldg(T.cen_id + m));
    stage_shared(L, T.lat + br.lat);
    const LatRef &F = T.ref[phase * T.nl + br.lat];
    centroid_body<R>(L, br.v, (R *)F.force, F.stamp, F.d_step, blockIdx.x - __ldg(T.cen_pre + m));
}

// ---- persistent batched step ----
__device__ __forceinline__ unsigned long long global_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Thread 0: waits until every item of kind k of lattice l in steps 0..upto
// of this launch has finished (count (upto + 1) * need).  Gives up, and
// marks the launch aborted, once the wait has lasted P.wait_ns, or when
// another block has aborted.  The acquire load orders the item's later
// loads after the awaited items' stores.
__device__ bool wait_kind(const PersistTables &P, int l, int k, int upto, unsigned long long t0) {
    const unsigned need = __ldg(P.need + l * kPKinds + k);
    if (upto < 0 || need == 0) return true;
    const unsigned target = (unsigned)(upto + 1) * need;
    const unsigned *ctr = P.done + l * kPKinds + k;
    for (;;) {
        if (ld_acquire(ctr) >= target) return true;
        if (*(volatile unsigned *)P.abort) return false;
        if ((long long)(global_ns() - t0) >= P.wait_ns) {
            atomicExch(P.abort, 1u);
            return false;
        }
        __nanosleep(100);
    }
}

// The items an item of kind k, lattice l, step s waits for: its lattice's
// earlier phases of the step, and the previous step's sweep.
__device__ bool wait_deps(const PersistTables &P, int k, int l, int s) {
    const unsigned long long t0 = global_ns();
    asm volatile("fence.acq_rel.gpu;" ::: "memory");  // an acquire even when nothing is awaited
    switch (k) {
        case kPMom: return wait_kind(P, l, kPSweep, s - 1, t0);
        case kPMls: return wait_kind(P, l, kPMom, s, t0);
        case kPMemb:
        case kPRf: return wait_kind(P, l, kPMls, s, t0);
        case kPRm: return wait_kind(P, l, kPRf, s, t0);
        case kPCen: return wait_kind(P, l, kPMemb, s, t0) && wait_kind(P, l, kPRm, s, t0);
        default:
            for (int j = kPMom; j < kPSweep; ++j)
                if (!wait_kind(P, l, j, s, t0)) return false;
            return wait_kind(P, l, kPSweep, s - 1, t0);
    }
}

// Several steps of every lattice of a batch in one launch: blocks take work
// items (support moments, MLS, structure updates, spreading, sweep tiles)
// in ticket order from a table that interleaves the lattices' chains (the
// host staggers them, so that each stretch of the queue mixes some
// lattices' sweeps with other lattices' IB phases), each item starting
// after the items it depends on (per-lattice completion counters).  A
// wait that exceeds its bound sets LBIB_ETIMEOUT on every lattice and ends
// the launch.
template <typename S, typename R, bool kOff32>
__global__ void __launch_bounds__(256, 4) kp_batch(BatchTables T, PersistTables P) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ Lattice L;
    __shared__ BodyRef br;
    __shared__ unsigned s_t[2];  // this item's ticket and the next one (taken early, double-buffered)
    __shared__ int s_ok;
    const unsigned total = (unsigned)P.nitems;
    if (threadIdx.x == 0) s_t[0] = atomicAdd(P.ticket, 1u);
    for (int k = 0;; k ^= 1) {
        __syncthreads();
        const unsigned t = s_t[k];
        if (t >= total) break;
        const int4 it = __ldg(P.items + t);
        const int kind = it.x & 0xff, s = it.x >> 8;
        const int phase = (P.phase0 + s) % 6;
        const int lat = kind == kPSweep ? it.y : __ldg(P.body_lat + it.y);
        if (threadIdx.x == 0) {
            s_ok = !*(volatile unsigned *)P.abort && wait_deps(P, kind, lat, s);
            if (!s_ok)
                for (int l = 0; l < T.nl; ++l) atomicCAS(T.ref[l].err, 0, kErrTimeout);
            s_t[k ^ 1] = atomicAdd(P.ticket, 1u);  // the next item's ticket, in flight during this one
        }
        // stage the lattice (and body) parameters; the barrier also
        // publishes s_ok
        {
            const uint32_t *srcL = reinterpret_cast<const uint32_t *>(T.lat + lat);
            uint32_t *dstL = reinterpret_cast<uint32_t *>(&L);
            for (int w = threadIdx.x; w < (int)(sizeof(Lattice) / 4); w += blockDim.x) dstL[w] = __ldg(srcL + w);
            if (kind != kPSweep) {
                const uint32_t *srcB = reinterpret_cast<const uint32_t *>(T.body + phase * T.nb + it.y);
                uint32_t *dstB = reinterpret_cast<uint32_t *>(&br);
                for (int w = threadIdx.x; w < (int)(sizeof(BodyRef) / 4); w += blockDim.x) dstB[w] = __ldg(srcB + w);
            }
        }
        __syncthreads();
        if (!s_ok) break;
        const LatRef &F = T.ref[phase * T.nl + lat];
        switch (kind) {
            case kPSweep: {
                const uint32_t step = F.stamp ? __ldcg(F.d_step) : 0u;
                const uint32_t seed = __ldcg(F.sr + F.parity);
                if (it.z == 0 && threadIdx.x == 0) F.sr[F.parity ^ 1] = seed + 1u;
                const int c0 = it.z * P.sweep_cells;
                const int c1 = min(c0 + P.sweep_cells, L.ncell);
                for (int c = c0 + (int)threadIdx.x; c < c1; c += blockDim.x) {
                    const int x = c % L.nx, yz = c / L.nx, y = yz % L.ny, z = yz / L.ny;
                    sweep_cell<S, R, kOff32, true>((const S *)F.fin, (S *)F.fout, (R *)F.force, F.stamp, step, L,
                                                   nullptr, x, y, z, seed);
                }
                break;
            }
            case kPMom:
                moments_body<S, R, true>((const S *)F.fin, L, br.v.bbox, br.v.bbox_next, (R *)F.mom,
                                         br.inc_step ? F.d_step : nullptr, it.z, it.w);
                break;
            case kPMls:
                mls_body<R, true, true>((const R *)F.mom, L, br.v, F.err,
                                        *reinterpret_cast<MlsSmem<R, true> *>(smem_raw), it.z, it.w);
                break;
            case kPMemb: membrane_body<R>(L, br.v, (R *)F.force, F.stamp, F.d_step, it.z); break;
            case kPRf: rigid_forces_body<R>(br.v, it.z, it.w); break;
            case kPRm: rigid_markers_body<R>(L, br.v, (R *)F.force, F.stamp, F.d_step, it.z); break;
            default: centroid_body<R>(L, br.v, (R *)F.force, F.stamp, F.d_step, it.z); break;
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();  // the item's stores (every thread's, ordered by the barrier) before its count
            atomicAdd(P.done + lat * kPKinds + kind, 1u);
        }
    }
}

template <typename S, typename R>
static cudaError_t persistent_t(const BatchTables &T, const PersistTables &P, int grid, cudaStream_t s) {
    if (T.sweep_off32)
        kp_batch<S, R, true><<<grid, 256, sizeof(MlsSmem<R, true>), s>>>(T, P);
    else
        kp_batch<S, R, false><<<grid, 256, sizeof(MlsSmem<R, true>), s>>>(T, P);
    return cudaGetLastError();
}

cudaError_t launch_batch_persistent(int prec, const BatchTables &T, const PersistTables &P, int grid,
                                    cudaStream_t s) {
    switch (prec) {
        case 0: return persistent_t<double, double>(T, P, grid, s);
        case 1: return persistent_t<float, float>(T, P, grid, s);
        case 2: return persistent_t<__half, float>(T, P, grid, s);
        default: return persistent_t<__nv_bfloat16, float>(T, P, grid, s);
    }
}

// Resident blocks per SM of the persistent kernel (its dynamic shared
// memory set), for the grid size.
template <typename S, typename R>
static int persistent_occ(bool off32) {
    int n = 0;
    const size_t smem = sizeof(MlsSmem<R, true>);
    if (off32) {
        cudaFuncSetAttribute(kp_batch<S, R, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kp_batch<S, R, true>, 256, smem);
    } else {
        cudaFuncSetAttribute(kp_batch<S, R, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, kp_batch<S, R, false>, 256, smem);
    }
    return n;
}

int batch_persistent_blocks_per_sm(int prec, bool off32) {
    switch (prec) {
        case 0: return persistent_occ<double, double>(off32);
        case 1: return persistent_occ<float, float>(off32);
        case 2: return persistent_occ<__half, float>(off32);
        default: return persistent_occ<__nv_bfloat16, float>(off32);
    }
}

template <typename S, typename R>
static cudaError_t batch_ib_t(const BatchTables &T, const BatchGrid &G, int phase, cudaStream_t s) {
    if (G.mom > 0) kb_moments<S, R><<<G.mom, 256, 0, s>>>(T, phase);
    if (G.mls > 0) kb_mls<R><<<G.mls, kMlsThreads, sizeof(MlsSmem<R>), s>>>(T, phase);
    if (G.memb > 0) kb_membrane<R><<<G.memb, 256, 0, s>>>(T, phase);
    if (G.rf > 0) kb_rigid_forces<R><<<G.rf, 256, 0, s>>>(T, phase);
    if (G.rm > 0) kb_rigid_markers<R><<<G.rm, 256, 0, s>>>(T, phase);
    if (G.cen > 0) kb_centroid_spread<R><<<G.cen, 256, 0, s>>>(T, phase);  // after the structure kernels
    return cudaGetLastError();
}

cudaError_t launch_batch_ib(int prec, const BatchTables &T, const BatchGrid &G, int phase, cudaStream_t s) {
    switch (prec) {
        case 0: return batch_ib_t<double, double>(T, G, phase, s);
        case 1: return batch_ib_t<float, float>(T, G, phase, s);
        case 2: return batch_ib_t<__half, float>(T, G, phase, s);
        default: return batch_ib_t<__nv_bfloat16, float>(T, G, phase, s);
    }
}

// ---- launchers ----
int mls_blocks(const BodyView &B) { return (B.nm + 2 * B.nt + kPts - 1) / kPts; }

// Grid of n blocks' work under a cap (0: none).
static int capped(int n, int cap) { return cap > 0 && cap < n ? cap : n; }

template <typename S, typename R>
static cudaError_t ib_front_t(const void *fin, const Lattice &L, const BodyView &B, void *mom, int nsm, int *err,
                              uint32_t *step_inc, int grid_cap, cudaStream_t s) {
    k_moments<S, R><<<2 * nsm, 256, 0, s>>>((const S *)fin, L, B.bbox, B.bbox_next, (R *)mom, step_inc);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    // the MLS kernel is scheduled while the moments kernel ends (measured:
    // about 2 us off the 96^3 capsule step; the same launch for the other
    // kernels of the step made it slower)
    const int nvb = mls_blocks(B);
    return launch_chained(k_mls<R>, dim3(capped(nvb, grid_cap)), dim3(kMlsThreads), sizeof(MlsSmem<R>), s,
                          (const R *)mom, L, B, err, nvb);
}

// Kernel attributes that must be set before the first launch (and before
// any stream capture): the MLS kernel's dynamic shared memory.
cudaError_t prepare_kernels() {
    cudaError_t e = cudaFuncSetAttribute(k_mls<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(MlsSmem<float>));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_mls<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(MlsSmem<double>));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kb_mls<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(MlsSmem<float>));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(kb_mls<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)sizeof(MlsSmem<double>));
    return e;
}

cudaError_t launch_ib_front(int prec, const void *fin, const Lattice &L, const BodyView &B, void *mom, int nsm,
                            int *err, uint32_t *step_inc, int grid_cap, cudaStream_t s) {
    switch (prec) {
        case 0: return ib_front_t<double, double>(fin, L, B, mom, nsm, err, step_inc, grid_cap, s);
        case 1: return ib_front_t<float, float>(fin, L, B, mom, nsm, err, step_inc, grid_cap, s);
        case 2: return ib_front_t<__half, float>(fin, L, B, mom, nsm, err, step_inc, grid_cap, s);
        default: return ib_front_t<__nv_bfloat16, float>(fin, L, B, mom, nsm, err, step_inc, grid_cap, s);
    }
}

static cudaError_t launch_centroid(int prec, const Lattice &L, const BodyView &B, void *force, uint32_t *stamp,
                                   const uint32_t *step, cudaStream_t s) {
    const unsigned g = (unsigned)((B.nt + 7) / 8);  // 8 warps (triangles) per block
    if (prec == 0)
        k_centroid_spread<double><<<g, 256, 0, s>>>(L, B, (double *)force, stamp, step);
    else
        k_centroid_spread<float><<<g, 256, 0, s>>>(L, B, (float *)force, stamp, step);
    return cudaGetLastError();
}

cudaError_t launch_membrane(int prec, const Lattice &L, const BodyView &B, void *force, uint32_t *stamp,
                            const uint32_t *step, int grid_cap, cudaStream_t s) {
    const int nvb = (B.nv + 7) / 8;  // 8 warps (vertices) per block
    const unsigned g = (unsigned)capped(nvb, grid_cap);
    if (prec == 0)
        k_membrane<double><<<g, 256, 0, s>>>(L, B, (double *)force, stamp, step, nvb);
    else
        k_membrane<float><<<g, 256, 0, s>>>(L, B, (float *)force, stamp, step, nvb);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !B.centroid) return e;
    return launch_centroid(prec, L, B, force, stamp, step, s);
}

cudaError_t launch_rigid(int prec, const Lattice &L, const BodyView &B, void *force, uint32_t *stamp,
                         const uint32_t *step, int grid_cap, cudaStream_t s) {
    const unsigned gf = (unsigned)((B.nt + 255) / 256);
    if (prec == 0)
        k_rigid_forces<double><<<gf, 256, 0, s>>>(B);
    else
        k_rigid_forces<float><<<gf, 256, 0, s>>>(B);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const int nvb = (B.nv + 7) / 8;
    const unsigned g = (unsigned)capped(nvb, grid_cap);
    if (prec == 0)
        k_rigid_markers<double><<<g, 256, 0, s>>>(L, B, (double *)force, stamp, step, nvb);
    else
        k_rigid_markers<float><<<g, 256, 0, s>>>(L, B, (float *)force, stamp, step, nvb);
    e = cudaGetLastError();
    if (e != cudaSuccess || !B.centroid) return e;
    return launch_centroid(prec, L, B, force, stamp, step, s);
}

}  // namespace lbib
