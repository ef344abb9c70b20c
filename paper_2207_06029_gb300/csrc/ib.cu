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

namespace lbib {

constexpr int kPts = 32;          // MLS points per block
constexpr int kMlsThreads = 128;  // 4 warps, 8 points each
constexpr double kAlpha = 0.3;    // Eq. (intKernel)
constexpr double kRw = 1.3;       // support size r_w (Sec. 2.2)
constexpr double kProbe = 1.2;    // probe length (Sec. 2.3)
constexpr int kBoxLo = 3, kBoxHi = 4;  // node margins that cover marker and probe supports

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
template <typename S, typename R>
__global__ void __launch_bounds__(256) k_moments(const S *__restrict__ fin, Lattice L, const int *__restrict__ box,
                                                 int *__restrict__ box_next, R *__restrict__ mom) {
    const int n[3] = {L.nx, L.ny, L.nz};
    int lo[3], ext[3];
    for (int a = 0; a < 3; ++a) {
        long long l = box[a], h = box[3 + a];
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
    if (blockIdx.x == 0 && threadIdx.x < 6) box_next[threadIdx.x] = threadIdx.x < 3 ? 0x7fffffff : (int)0x80000000;
    const int total = ext[0] * ext[1] * ext[2];
    const int nxy = L.nx * L.ny;
    const long long st = L.stride;
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x) {
        int c[3] = {lo[0] + k % ext[0], lo[1] + (k / ext[0]) % ext[1], lo[2] + k / (ext[0] * ext[1])};
        int cm[3], cp[3];
        for (int a = 0; a < 3; ++a) {
            if (L.bc[a] == kPeriodic) c[a] = ((c[a] % n[a]) + n[a]) % n[a];
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
            const R gi = Pop<S, R>::ld(fin + (long long)i * st + (sx + L.nx * sy + nxy * sz));
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
        mom[node] = drho;
        mom[st + node] = (jx + R(0.5 * L.gext[0])) / rho;
        mom[2 * st + node] = (jy + R(0.5 * L.gext[1])) / rho;
        mom[3 * st + node] = (jz + R(0.5 * L.gext[2])) / rho;
    }
}

template <typename R>
struct MlsSmem {
    R W[kPts][27];
    R d[kPts][27][3];
    R rho[kPts][27];
    R u[kPts][27][3];
    R nrm[kPts][3];
    double vol[kPts];
    double A[kPts][10];
    double Ai[kPts][16];
};

// Inverse of a symmetric positive definite 4x4 matrix given by its upper
// triangle (00,01,02,03,11,12,13,22,23,33), through its Cholesky factor.
__device__ bool spd_inverse4(const double *a, double *inv) {
    double M[4][4];
    M[0][0] = a[0]; M[0][1] = M[1][0] = a[1]; M[0][2] = M[2][0] = a[2]; M[0][3] = M[3][0] = a[3];
    M[1][1] = a[4]; M[1][2] = M[2][1] = a[5]; M[1][3] = M[3][1] = a[6];
    M[2][2] = a[7]; M[2][3] = M[3][2] = a[8]; M[3][3] = a[9];
    double Lw[4][4] = {{0}}, Li[4][4] = {{0}};
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        double s = M[j][j];
#pragma unroll
        for (int k = 0; k < j; ++k) s -= Lw[j][k] * Lw[j][k];
        if (!(s > 0.0)) return false;
        Lw[j][j] = sqrt(s);
#pragma unroll
        for (int i = j + 1; i < 4; ++i) {
            double t = M[i][j];
#pragma unroll
            for (int k = 0; k < j; ++k) t -= Lw[i][k] * Lw[j][k];
            Lw[i][j] = t / Lw[j][j];
        }
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        Li[i][i] = 1.0 / Lw[i][i];
#pragma unroll
        for (int j = 0; j < i; ++j) {
            double t = 0.0;
#pragma unroll
            for (int k = j; k < i; ++k) t += Lw[i][k] * Li[k][j];
            Li[i][j] = -t * Li[i][i];
        }
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            double t = 0.0;
#pragma unroll
            for (int k = (r > c ? r : c); k < 4; ++k) t += Li[k][r] * Li[k][c];
            inv[4 * r + c] = t;
        }
    return true;
}

// Triangle geometry in arithmetic R from double positions: unit normal,
// area, centroid (double) and the volume term (x_0 - o) . (e1 x e2).
template <typename R>
__device__ __forceinline__ void tri_geometry(const double *X, const int *t, const double *o, R *n, R &area,
                                             double *cen, double &vol6) {
    const int i0 = t[0], i1 = t[1], i2 = t[2];
    const double x0[3] = {X[3 * i0], X[3 * i0 + 1], X[3 * i0 + 2]};
    const R e1[3] = {R(X[3 * i1] - x0[0]), R(X[3 * i1 + 1] - x0[1]), R(X[3 * i1 + 2] - x0[2])};
    const R e2[3] = {R(X[3 * i2] - x0[0]), R(X[3 * i2 + 1] - x0[1]), R(X[3 * i2 + 2] - x0[2])};
    const R N[3] = {e1[1] * e2[2] - e1[2] * e2[1], e1[2] * e2[0] - e1[0] * e2[2], e1[0] * e2[1] - e1[1] * e2[0]};
    const R nn = sqrt(N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
    area = R(0.5) * nn;
    for (int a = 0; a < 3; ++a) {
        n[a] = N[a] / nn;
        cen[a] = x0[a] + (double)((e1[a] + e2[a]) / R(3));
    }
    vol6 = (x0[0] - o[0]) * (double)N[0] + (x0[1] - o[1]) * (double)N[1] + (x0[2] - o[2]) * (double)N[2];
}

// One warp per point, 32 points per block.  Points 0..nv-1 are the markers;
// point nv + 2t + side is the probe of triangle t on the outer (side 0) or
// inner (side 1) face.
//  phase 1: support block, weights (the r_k <= 1 decision bit-exact in
//           FP64), node moments, moment matrix A (warp reduction);
//  phase 2: warp 0 inverts the 32 matrices in FP64, one lane each;
//  phase 3: shape functions psi_k = W_k A^-1 p_k; markers interpolate U and
//           keep phi = psi[0] for spreading; probes fit rho and u and store
//           pressure and traction.
template <typename R>
__global__ void __launch_bounds__(kMlsThreads) k_mls(const R *__restrict__ mom, Lattice L, BodyView B,
                                                     int *err) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    MlsSmem<R> &sm = *reinterpret_cast<MlsSmem<R> *>(smem_raw);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int npts = B.nv + 2 * B.nt;
    const int p0 = blockIdx.x * kPts;
    const long long st = L.stride;
    const int nxy = L.nx * L.ny;
    const int n[3] = {L.nx, L.ny, L.nz};
    if (threadIdx.x < kPts) sm.vol[threadIdx.x] = 0.0;
    __syncthreads();

    // ---------------- phase 1 ----------------
    for (int j = 0; j < kPts / 4; ++j) {
        const int lp = warp * (kPts / 4) + j;
        const int p = p0 + lp;
        if (p >= npts) break;
        double P[3];
        if (p < B.nv) {
            P[0] = B.X[3 * p];
            P[1] = B.X[3 * p + 1];
            P[2] = B.X[3 * p + 2];
        } else {
            const int t = (p - B.nv) >> 1, side = (p - B.nv) & 1;
            R nr[3], area;
            double cen[3], vol6;
            tri_geometry<R>(B.X, B.tri + 3 * t, B.origin, nr, area, cen, vol6);
            const double sg = side ? -kProbe : kProbe;
            for (int a = 0; a < 3; ++a) P[a] = cen[a] + sg * (double)nr[a];
            if (lane == 0) {
                sm.nrm[lp][0] = nr[0];
                sm.nrm[lp][1] = nr[1];
                sm.nrm[lp][2] = nr[2];
                if (side == 0) {
                    double *tg = B.tri_geo + 8 * t;
                    tg[0] = nr[0];
                    tg[1] = nr[1];
                    tg[2] = nr[2];
                    tg[3] = area;
                    tg[4] = cen[0];
                    tg[5] = cen[1];
                    tg[6] = cen[2];
                    tg[7] = vol6;
                    sm.vol[lp] = vol6;
                }
            }
        }
        // nearest node and wall check (supports stay off wall nodes)
        int base[3];
        bool bad = false;
        for (int a = 0; a < 3; ++a) {
            base[a] = (int)floor(P[a] + 0.5);
            if (L.bc[a] == kWall && (base[a] - 1 < 1 || base[a] + 1 > n[a] - 2)) {
                bad = true;
                base[a] = base[a] < 2 ? 2 : (base[a] > n[a] - 3 ? n[a] - 3 : base[a]);
            }
        }
        if (bad && lane == 0) atomicCAS(err, 0, -5);
        R W = R(0), dk[3] = {R(0), R(0), R(0)};
        if (lane < 27) {
            const int dd[3] = {lane % 3 - 1, (lane / 3) % 3 - 1, lane / 9 - 1};
            int cw[3];
            double dx[3];
            for (int a = 0; a < 3; ++a) {
                const int c = base[a] + dd[a];
                dx[a] = (double)c - P[a];
                dk[a] = R(dx[a]);
                cw[a] = L.bc[a] == kPeriodic ? ((c % n[a]) + n[a]) % n[a] : c;
            }
            // |x_k - X|^2 rounded exactly as the plain sum of squares, so the
            // cut-off r_k <= 1 of Eq. (intKernel) is decided bit for bit
            const double dist2 = __dadd_rn(__dadd_rn(__dmul_rn(dx[0], dx[0]), __dmul_rn(dx[1], dx[1])),
                                           __dmul_rn(dx[2], dx[2]));
            if (dist2 <= L.dist2_cut) {
                const R r = sqrt(R(dist2)) / R(kRw);
                W = exp(-(r / R(kAlpha)) * (r / R(kAlpha)));
            }
            const int node = cw[0] + L.nx * cw[1] + nxy * cw[2];
            if (p < B.nv) B.node[27 * p + lane] = node;
            sm.W[lp][lane] = W;
            sm.rho[lp][lane] = mom[node];
            sm.u[lp][lane][0] = mom[st + node];
            sm.u[lp][lane][1] = mom[2 * st + node];
            sm.u[lp][lane][2] = mom[3 * st + node];
            for (int a = 0; a < 3; ++a) sm.d[lp][lane][a] = dk[a];
        }
        // moment matrix A = sum W p p^T, p = (1, x_k - X)
        R a10[10] = {W, W * dk[0], W * dk[1], W * dk[2], W * dk[0] * dk[0], W * dk[0] * dk[1],
                     W * dk[0] * dk[2], W * dk[1] * dk[1], W * dk[1] * dk[2], W * dk[2] * dk[2]};
#pragma unroll
        for (int q = 0; q < 10; ++q) a10[q] = warp_sum(a10[q]);
        if (lane == 0)
            for (int q = 0; q < 10; ++q) sm.A[lp][q] = (double)a10[q];
    }
    __syncthreads();

    // ---------------- phase 2: FP64 solves, one lane per point ----------------
    if (warp == 0 && p0 + lane < npts) {
        if (!spd_inverse4(sm.A[lane], sm.Ai[lane])) atomicCAS(err, 0, -1);
    }
    if (threadIdx.x == 32 && B.vol_part) {  // fixed-order partial of the enclosed volume
        double s = 0.0;
        for (int k = 0; k < kPts; ++k) s += sm.vol[k];
        B.vol_part[blockIdx.x] = s;
    }
    __syncthreads();

    // ---------------- phase 3 ----------------
    const R nu = R((L.tau - 0.5) / 3.0);
    for (int j = 0; j < kPts / 4; ++j) {
        const int lp = warp * (kPts / 4) + j;
        const int p = p0 + lp;
        if (p >= npts) break;
        R W = R(0), d0 = R(0), d1 = R(0), d2 = R(0), rk = R(0), u0 = R(0), u1 = R(0), u2 = R(0);
        if (lane < 27) {
            W = sm.W[lp][lane];
            d0 = sm.d[lp][lane][0];
            d1 = sm.d[lp][lane][1];
            d2 = sm.d[lp][lane][2];
            rk = sm.rho[lp][lane];
            u0 = sm.u[lp][lane][0];
            u1 = sm.u[lp][lane][1];
            u2 = sm.u[lp][lane][2];
        }
        const double *Ai = sm.Ai[lp];
        if (p < B.nv) {
            const R phi = W * (R(Ai[0]) + R(Ai[1]) * d0 + R(Ai[2]) * d1 + R(Ai[3]) * d2);
            if (lane < 27) B.phi[27 * p + lane] = (double)phi;
            const R U0 = warp_sum(phi * u0), U1 = warp_sum(phi * u1), U2 = warp_sum(phi * u2);
            if (lane == 0) {
                B.U[3 * p] = U0;
                B.U[3 * p + 1] = U1;
                B.U[3 * p + 2] = U2;
            }
        } else {
            R psi[4];
#pragma unroll
            for (int i = 0; i < 4; ++i)
                psi[i] = W * (R(Ai[4 * i]) + R(Ai[4 * i + 1]) * d0 + R(Ai[4 * i + 2]) * d1 + R(Ai[4 * i + 3]) * d2);
            R fit[16];
#pragma unroll
            for (int i = 0; i < 4; ++i) {
                fit[i] = warp_sum(psi[i] * rk);
                fit[4 + i] = warp_sum(psi[i] * u0);
                fit[8 + i] = warp_sum(psi[i] * u1);
                fit[12 + i] = warp_sum(psi[i] * u2);
            }
            if (lane == 0) {
                const int t = (p - B.nv) >> 1, side = (p - B.nv) & 1;
                const R rho = R(1) + fit[0];
                // grad u: du_j/dx_m = fit[4 + 4j + 1 + m]
                R tn[3];
#pragma unroll
                for (int jj = 0; jj < 3; ++jj) {
                    R acc = R(0);
#pragma unroll
                    for (int m = 0; m < 3; ++m)
                        acc += rho * nu * (fit[4 + 4 * jj + 1 + m] + fit[4 + 4 * m + 1 + jj]) * sm.nrm[lp][m];
                    tn[jj] = acc;
                }
                double *pr = B.probe + 8 * t + 4 * side;
                pr[0] = (1.0 + (double)fit[0]) / 3.0;
                pr[1] = tn[0];
                pr[2] = tn[1];
                pr[3] = tn[2];
            }
        }
    }
}

// Hydrodynamic force on triangle t from its two probes (Eqs. hydroForP,
// hydroForNu): F = [-(p+ - p-) n + (tau+ - tau-) . n] A.
__device__ __forceinline__ void tri_hydro(const BodyView &B, int t, double *F) {
    const double *tg = B.tri_geo + 8 * t;
    const double *pp = B.probe + 8 * t, *pm = pp + 4;
    const double A = tg[3];
    for (int a = 0; a < 3; ++a) F[a] = (-(pp[0] - pm[0]) * tg[a] + (pp[1 + a] - pm[1 + a])) * A;
}

// Lanes 0..26 of a warp add c phi_k F to the force field at the support
// nodes of marker v; the lanes of the 8 block corners flag their tiles.
template <typename R>
__device__ __forceinline__ void spread_warp(const Lattice &L, const BodyView &B, int v, int lane, double c,
                                            const double *Fl, R *__restrict__ force, uint32_t *stamp,
                                            uint32_t step) {
    if (lane >= 27) return;
    const long long st = L.stride;
    const int node = B.node[27 * v + lane];
    const double w = c * B.phi[27 * v + lane];
    atomicAdd(force + node, R(w * Fl[0]));
    atomicAdd(force + st + node, R(w * Fl[1]));
    atomicAdd(force + 2 * st + node, R(w * Fl[2]));
    if (lane == 0 || lane == 2 || lane == 6 || lane == 8 || lane == 18 || lane == 20 || lane == 24 || lane == 26) {
        const int x = node % L.nx, yz = node / L.nx, y = yz % L.ny, z = yz / L.ny;
        stamp[(x >> 3) + L.ntx * ((y >> 3) + L.nty * (z >> 3))] = step;
    }
}

// Grows the node box of level n+1 by one marker position.
__device__ __forceinline__ void box_add(int *box, const double *x) {
    for (int a = 0; a < 3; ++a) {
        const int c = (int)floor(x[a]);
        atomicMin(box + a, c - kBoxLo);
        atomicMax(box + 3 + a, c + kBoxHi);
    }
}

// Membrane vertex update, one warp per vertex: spring (Eq. strainFor),
// bending (gradient of k_b[1 - cos(theta - theta0)], reading of Eq. bendFor),
// volume penalty (restoring reading of Eq. volFor) and element hydrodynamic
// forces shared 1/3 per vertex (Eq. newtonSoft), with the lanes sharing the
// incident hinges and triangles; Verlet positions (Eqs. verletPos,
// verletVel); boundary velocity U_b = U + F/m_v dt; the Lagrangian force
// F_l = U_b - U spread with c_l = A_l (Eq. bodyforce).
template <typename R>
__global__ void __launch_bounds__(256) k_membrane(Lattice L, BodyView B, R *__restrict__ force,
                                                  uint32_t *__restrict__ stamp, uint32_t step) {
    __shared__ double sV;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 32) {
        double s = 0.0;
        for (int i = lane; i < B.nvol_part; i += 32) s += B.vol_part[i];
        s = warp_sum(s);
        if (lane == 0) sV = s / 6.0;
    }
    __syncthreads();
    const double V = sV;
    const int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (v >= B.nv) return;
    const double *X = B.X;
    R F[3] = {R(0), R(0), R(0)};
    for (int q = B.vh_ptr[v] + lane; q < B.vh_ptr[v + 1]; q += 32) {
        const int code = B.vh_list[q];
        const int h = code >> 2, role = code & 3;
        const int4 H = B.hinge[h];
        const double xa[3] = {X[3 * H.x], X[3 * H.x + 1], X[3 * H.x + 2]};
        R e[3], ac[3], ad[3];
        for (int a = 0; a < 3; ++a) {
            e[a] = R(X[3 * H.y + a] - xa[a]);
            ac[a] = R(X[3 * H.z + a] - xa[a]);
            ad[a] = R(X[3 * H.w + a] - xa[a]);
        }
        const R le2 = e[0] * e[0] + e[1] * e[1] + e[2] * e[2];
        const R le = sqrt(le2);
        if (role < 2) {
            // F_a = -k (l - l0) (x_a - x_b)/l = k (l - l0) e / l, F_b = -F_a
            const R c = R(B.ks[h]) * (le - R(B.l0[h])) / le;
            const R sg = role == 0 ? R(1) : R(-1);
            for (int a = 0; a < 3; ++a) F[a] += sg * c * e[a];
        }
        const R N1[3] = {e[1] * ac[2] - e[2] * ac[1], e[2] * ac[0] - e[0] * ac[2], e[0] * ac[1] - e[1] * ac[0]};
        const R N2[3] = {ad[1] * e[2] - ad[2] * e[1], ad[2] * e[0] - ad[0] * e[2], ad[0] * e[1] - ad[1] * e[0]};
        const R l1 = sqrt(N1[0] * N1[0] + N1[1] * N1[1] + N1[2] * N1[2]);
        const R l2 = sqrt(N2[0] * N2[0] + N2[1] * N2[1] + N2[2] * N2[2]);
        R n1[3], n2[3];
        for (int a = 0; a < 3; ++a) {
            n1[a] = N1[a] / l1;
            n2[a] = N2[a] / l2;
        }
        const R cx[3] = {n1[1] * n2[2] - n1[2] * n2[1], n1[2] * n2[0] - n1[0] * n2[2], n1[0] * n2[1] - n1[1] * n2[0]};
        const R theta = atan2((cx[0] * e[0] + cx[1] * e[1] + cx[2] * e[2]) / le,
                              n1[0] * n2[0] + n1[1] * n2[1] + n1[2] * n2[2]);
        const R dth = theta - R(B.theta0[h]);
        const R dE = B.bend_variant ? R(B.kb[h]) * dth : R(B.kb[h]) * sin(dth);
        const R h1 = l1 / le, h2 = l2 / le;
        const R tc = (ac[0] * e[0] + ac[1] * e[1] + ac[2] * e[2]) / le2;
        const R td = (ad[0] * e[0] + ad[1] * e[1] + ad[2] * e[2]) / le2;
        R c1, c2;  // dtheta/dx = c1 n1/h1 + c2 n2/h2
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
        for (int a = 0; a < 3; ++a) F[a] -= dE * (c1 * n1[a] / h1 + c2 * n2[a] / h2);
    }
    // element terms: volume penalty and hydrodynamic force, 1/3 per vertex
    const R cv = R(B.kv * (1.0 - V / B.V0));
    double Al = 0.0;
    for (int q = B.vt_ptr[v] + lane; q < B.vt_ptr[v + 1]; q += 32) {
        const int t = B.vt_list[q] / 3;
        const double *tg = B.tri_geo + 8 * t;
        Al += tg[3] / 3.0;
        double Fh[3];
        tri_hydro(B, t, Fh);
        for (int a = 0; a < 3; ++a) F[a] += cv * R(tg[a]) * R(tg[3]) / R(3) + R(Fh[a] / 3.0);
    }
    for (int a = 0; a < 3; ++a) F[a] = warp_sum(F[a]);
    Al = warp_sum(Al);
    // Newton (Eq. newtonSoft) and Verlet (Eqs. verletPos, verletVel), dt = 1
    double Fl[3];
    for (int a = 0; a < 3; ++a) {
        const double acc = (double)F[a] / B.mv;
        const double U = B.U[3 * v + a];
        const double Ub = U + acc;
        Fl[a] = Ub - U;
        if (lane == 0) {
            const double x = X[3 * v + a], xp = B.Xprev[3 * v + a];
            const double xt = x + U + 0.5 * acc;
            const double ubdf = 1.5 * xt - 2.0 * x + 0.5 * xp;
            B.Xnew[3 * v + a] = x + ubdf + 0.5 * acc;
            B.Ub[3 * v + a] = Ub;
            B.Fl[3 * v + a] = Fl[a];
        }
    }
    if (lane == 0) {
        double xn[3] = {B.Xnew[3 * v], B.Xnew[3 * v + 1], B.Xnew[3 * v + 2]};
        box_add(B.bbox_next, xn);
    }
    spread_warp<R>(L, B, v, lane, Al, Fl, force, stamp, step);
}

// Rigid body, one block: total force and moment of the element stresses,
// gravity minus buoyancy, F = m du/dt and M = I dw/dt with I in the world
// frame, second-order backward velocities (Eqs. linearVelRig,
// angularVelRig), centre and orientation advanced with the new velocities.
__global__ void __launch_bounds__(256) k_rigid_update(BodyView B) {
    __shared__ double red[6][256];
    double *S = B.rstate;
    const double xc[3] = {S[RigidState::XC], S[RigidState::XC + 1], S[RigidState::XC + 2]};
    double f[3] = {0, 0, 0}, m[3] = {0, 0, 0};
    for (int t = threadIdx.x; t < B.nt; t += blockDim.x) {
        double Fh[3];
        tri_hydro(B, t, Fh);
        const double *tg = B.tri_geo + 8 * t;
        const double r[3] = {tg[4] - xc[0], tg[5] - xc[1], tg[6] - xc[2]};
        f[0] += Fh[0];
        f[1] += Fh[1];
        f[2] += Fh[2];
        m[0] += r[1] * Fh[2] - r[2] * Fh[1];
        m[1] += r[2] * Fh[0] - r[0] * Fh[2];
        m[2] += r[0] * Fh[1] - r[1] * Fh[0];
    }
    for (int a = 0; a < 3; ++a) {
        red[a][threadIdx.x] = f[a];
        red[3 + a][threadIdx.x] = m[a];
    }
    __syncthreads();
    for (int h = blockDim.x / 2; h > 0; h >>= 1) {
        if (threadIdx.x < h)
            for (int q = 0; q < 6; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + h];
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    double F[3], M[3];
    for (int a = 0; a < 3; ++a) {
        F[a] = red[a][0] + (S[RigidState::DENS] - 1.0) * S[RigidState::VOL] * S[RigidState::GRAV + a];
        M[a] = red[3 + a][0];
    }
    const double *q = S + RigidState::Q4;
    const double *Ib = S + RigidState::IB;
    double R[9];
    {
        const double w = q[0], x = q[1], y = q[2], z = q[3];
        R[0] = 1 - 2 * (y * y + z * z); R[1] = 2 * (x * y - w * z); R[2] = 2 * (x * z + w * y);
        R[3] = 2 * (x * y + w * z); R[4] = 1 - 2 * (x * x + z * z); R[5] = 2 * (y * z - w * x);
        R[6] = 2 * (x * z - w * y); R[7] = 2 * (y * z + w * x); R[8] = 1 - 2 * (x * x + y * y);
    }
    double T[9], Iw[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += R[3 * i + k] * Ib[3 * k + j];
            T[3 * i + j] = acc;
        }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int k = 0; k < 3; ++k) acc += T[3 * i + k] * R[3 * j + k];
            Iw[3 * i + j] = acc;
        }
    const double det = Iw[0] * (Iw[4] * Iw[8] - Iw[5] * Iw[7]) - Iw[1] * (Iw[3] * Iw[8] - Iw[5] * Iw[6]) +
                       Iw[2] * (Iw[3] * Iw[7] - Iw[4] * Iw[6]);
    double Ii[9];
    Ii[0] = (Iw[4] * Iw[8] - Iw[5] * Iw[7]) / det;
    Ii[1] = (Iw[2] * Iw[7] - Iw[1] * Iw[8]) / det;
    Ii[2] = (Iw[1] * Iw[5] - Iw[2] * Iw[4]) / det;
    Ii[3] = (Iw[5] * Iw[6] - Iw[3] * Iw[8]) / det;
    Ii[4] = (Iw[0] * Iw[8] - Iw[2] * Iw[6]) / det;
    Ii[5] = (Iw[2] * Iw[3] - Iw[0] * Iw[5]) / det;
    Ii[6] = (Iw[3] * Iw[7] - Iw[4] * Iw[6]) / det;
    Ii[7] = (Iw[1] * Iw[6] - Iw[0] * Iw[7]) / det;
    Ii[8] = (Iw[0] * Iw[4] - Iw[1] * Iw[3]) / det;
    double un[3], wn[3];
    for (int a = 0; a < 3; ++a) {
        const double udot = F[a] / S[RigidState::MASS];
        const double wdot = Ii[3 * a] * M[0] + Ii[3 * a + 1] * M[1] + Ii[3 * a + 2] * M[2];
        un[a] = 2.0 / 3.0 * (2.0 * S[RigidState::U + a] - 0.5 * S[RigidState::UP + a] + udot);
        wn[a] = 2.0 / 3.0 * (2.0 * S[RigidState::W + a] - 0.5 * S[RigidState::WP + a] + wdot);
    }
    for (int a = 0; a < 3; ++a) {
        S[RigidState::XC_OLD + a] = xc[a];
        S[RigidState::XC + a] = xc[a] + un[a];
        S[RigidState::UP + a] = S[RigidState::U + a];
        S[RigidState::U + a] = un[a];
        S[RigidState::WP + a] = S[RigidState::W + a];
        S[RigidState::W + a] = wn[a];
    }
    const double wl = sqrt(wn[0] * wn[0] + wn[1] * wn[1] + wn[2] * wn[2]);
    double qn[4] = {q[0], q[1], q[2], q[3]};
    if (wl > 0.0) {
        const double c = cos(0.5 * wl), s = sin(0.5 * wl);
        const double dq[4] = {c, s * wn[0] / wl, s * wn[1] / wl, s * wn[2] / wl};
        qn[0] = dq[0] * q[0] - dq[1] * q[1] - dq[2] * q[2] - dq[3] * q[3];
        qn[1] = dq[0] * q[1] + dq[1] * q[0] + dq[2] * q[3] - dq[3] * q[2];
        qn[2] = dq[0] * q[2] - dq[1] * q[3] + dq[2] * q[0] + dq[3] * q[1];
        qn[3] = dq[0] * q[3] + dq[1] * q[2] - dq[2] * q[1] + dq[3] * q[0];
        const double qq = sqrt(qn[0] * qn[0] + qn[1] * qn[1] + qn[2] * qn[2] + qn[3] * qn[3]);
        for (int k = 0; k < 4; ++k) qn[k] /= qq;
    }
    for (int k = 0; k < 4; ++k) S[RigidState::Q4 + k] = qn[k];
    {
        const double w = qn[0], x = qn[1], y = qn[2], z = qn[3];
        double *Rn = S + RigidState::ROT;
        Rn[0] = 1 - 2 * (y * y + z * z); Rn[1] = 2 * (x * y - w * z); Rn[2] = 2 * (x * z + w * y);
        Rn[3] = 2 * (x * y + w * z); Rn[4] = 1 - 2 * (x * x + z * z); Rn[5] = 2 * (y * z - w * x);
        Rn[6] = 2 * (x * z - w * y); Rn[7] = 2 * (y * z + w * x); Rn[8] = 1 - 2 * (x * x + y * y);
    }
}

// Rigid markers, one warp each: boundary velocity u + w x (X - x_c) of
// level n, IB force and spreading, then the markers of level n+1.
template <typename R>
__global__ void __launch_bounds__(256) k_rigid_markers(Lattice L, BodyView B, R *__restrict__ force,
                                                       uint32_t *__restrict__ stamp, uint32_t step) {
    const int lane = threadIdx.x & 31;
    const int v = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (v >= B.nv) return;
    const double *S = B.rstate;
    const double *un = S + RigidState::U, *wn = S + RigidState::W, *xo = S + RigidState::XC_OLD;
    const double *xc = S + RigidState::XC, *Rn = S + RigidState::ROT;
    double Al = 0.0;
    for (int q = B.vt_ptr[v] + lane; q < B.vt_ptr[v + 1]; q += 32) Al += B.tri_geo[8 * (B.vt_list[q] / 3) + 3] / 3.0;
    Al = warp_sum(Al);
    const double r[3] = {B.X[3 * v] - xo[0], B.X[3 * v + 1] - xo[1], B.X[3 * v + 2] - xo[2]};
    const double wxr[3] = {wn[1] * r[2] - wn[2] * r[1], wn[2] * r[0] - wn[0] * r[2], wn[0] * r[1] - wn[1] * r[0]};
    double Fl[3];
    for (int a = 0; a < 3; ++a) {
        const double ub = un[a] + wxr[a];
        Fl[a] = ub - B.U[3 * v + a];
        if (lane == 0) {
            B.Ub[3 * v + a] = ub;
            B.Fl[3 * v + a] = Fl[a];
        }
    }
    if (lane == 0) {
        const double *xb = B.Xbody + 3 * v;
        double xn[3];
        for (int a = 0; a < 3; ++a) {
            xn[a] = xc[a] + Rn[3 * a] * xb[0] + Rn[3 * a + 1] * xb[1] + Rn[3 * a + 2] * xb[2];
            B.Xnew[3 * v + a] = xn[a];
        }
        box_add(B.bbox_next, xn);
    }
    spread_warp<R>(L, B, v, lane, Al, Fl, force, stamp, step);
}

// ---- launchers ----
int mls_blocks(const BodyView &B) { return (B.nv + 2 * B.nt + kPts - 1) / kPts; }

template <typename S, typename R>
static cudaError_t ib_front_t(const void *fin, const Lattice &L, const BodyView &B, void *mom, int nsm, int *err,
                              cudaStream_t s) {
    k_moments<S, R><<<4 * nsm, 256, 0, s>>>((const S *)fin, L, B.bbox, B.bbox_next, (R *)mom);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const size_t smem = sizeof(MlsSmem<R>);
    static bool attr_set = false;
    if (!attr_set) {
        e = cudaFuncSetAttribute(k_mls<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    k_mls<R><<<mls_blocks(B), kMlsThreads, smem, s>>>((const R *)mom, L, B, err);
    return cudaGetLastError();
}

cudaError_t launch_ib_front(int prec, const void *fin, const Lattice &L, const BodyView &B, void *mom, int nsm,
                            int *err, cudaStream_t s) {
    switch (prec) {
        case 0: return ib_front_t<double, double>(fin, L, B, mom, nsm, err, s);
        case 1: return ib_front_t<float, float>(fin, L, B, mom, nsm, err, s);
        case 2: return ib_front_t<__half, float>(fin, L, B, mom, nsm, err, s);
        default: return ib_front_t<__nv_bfloat16, float>(fin, L, B, mom, nsm, err, s);
    }
}

cudaError_t launch_membrane(int prec, const Lattice &L, const BodyView &B, void *force, uint32_t *stamp,
                            uint32_t step, cudaStream_t s) {
    const unsigned g = (unsigned)((B.nv + 7) / 8);  // 8 warps (vertices) per block
    if (prec == 0)
        k_membrane<double><<<g, 256, 0, s>>>(L, B, (double *)force, stamp, step);
    else
        k_membrane<float><<<g, 256, 0, s>>>(L, B, (float *)force, stamp, step);
    return cudaGetLastError();
}

cudaError_t launch_rigid(int prec, const Lattice &L, const BodyView &B, void *force, uint32_t *stamp,
                         uint32_t step, cudaStream_t s) {
    k_rigid_update<<<1, 256, 0, s>>>(B);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    const unsigned g = (unsigned)((B.nv + 7) / 8);
    if (prec == 0)
        k_rigid_markers<double><<<g, 256, 0, s>>>(L, B, (double *)force, stamp, step);
    else
        k_rigid_markers<float><<<g, 256, 0, s>>>(L, B, (float *)force, stamp, step);
    return cudaGetLastError();
}

}  // namespace lbib
