// Device-side definitions shared by the kernels of liblbib: the D3Q19
// molecule, storage conversions and the views of lattice and body state
// that kernels receive by value.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace lbib {

constexpr int Q = 19;
constexpr int kPeriodic = 0;
constexpr int kWall = 1;
constexpr int kTile = 8;  // edge of the cubic tiles that carry an IB-force flag

// Programmatic dependent launch (sm_90 and later).  A kernel launched with
// programmatic stream serialization may be scheduled once every block of
// its predecessor in the stream has called chain_release() (or ended); it
// calls chain_wait() before its first global-memory access, which returns
// when the predecessor has completed and its writes are visible.  Without
// that launch attribute chain_wait() returns at once.
__device__ __forceinline__ void chain_release() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }
__device__ __forceinline__ void chain_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// D3Q19 velocities, columns of the matrix of Eq. (e_i), Sec. 2.1.
__host__ __device__ constexpr int ex(int i) {
    return (i == 1 || i == 7 || i == 8 || i == 9 || i == 10) ? 1
           : (i == 2 || i == 11 || i == 12 || i == 13 || i == 14) ? -1
                                                                  : 0;
}
__host__ __device__ constexpr int ey(int i) {
    return (i == 3 || i == 7 || i == 11 || i == 15 || i == 16) ? 1
           : (i == 4 || i == 8 || i == 12 || i == 17 || i == 18) ? -1
                                                                 : 0;
}
__host__ __device__ constexpr int ez(int i) {
    return (i == 5 || i == 9 || i == 13 || i == 15 || i == 17) ? 1
           : (i == 6 || i == 10 || i == 14 || i == 16 || i == 18) ? -1
                                                                  : 0;
}
__host__ __device__ constexpr int ecomp(int i, int a) { return a == 0 ? ex(i) : a == 1 ? ey(i) : ez(i); }
// opposite direction: e_opp(i) = -e_i
__host__ __device__ constexpr int opp(int i) {
    return i == 0 ? 0 : i <= 6 ? (i % 2 ? i + 1 : i - 1) : i == 7 ? 12 : i == 8 ? 11 : i == 9 ? 14 : i == 10 ? 13
         : i == 11 ? 8 : i == 12 ? 7 : i == 13 ? 10 : i == 14 ? 9 : i == 15 ? 18 : i == 16 ? 17 : i == 17 ? 16 : 15;
}
// weights: 1/3, 1/18 (axis), 1/36 (diagonals), stated after Eq. (eqfunc)
template <typename R>
__host__ __device__ constexpr R wq(int i) {
    return i == 0 ? R(1) / R(3) : i <= 6 ? R(1) / R(18) : R(1) / R(36);
}

constexpr bool lattice_is_consistent() {
    for (int i = 0; i < Q; ++i) {
        int o = opp(i);
        if (ex(o) != -ex(i) || ey(o) != -ey(i) || ez(o) != -ez(i)) return false;
        int n2 = ex(i) * ex(i) + ey(i) * ey(i) + ez(i) * ez(i);
        if ((i == 0) != (n2 == 0) || (i >= 1 && i <= 6) != (n2 == 1)) return false;
    }
    return true;
}
static_assert(lattice_is_consistent(), "D3Q19 table");

// Loads of data that a launch never writes take the read-only path (__ldg).
// A launch that reads data other blocks of the same launch wrote (the
// persistent batched step: one work item's populations, flags and moments
// are written by earlier items) must not use that path, which lies outside
// the memory model: with kCG it issues plain weak loads (ld.global.ca,
// cached in L1 like the read-only path), which the memory model orders
// after the item's acquire of its dependency counter and the block barrier
// that follows it, so they see the awaited items' stores.  Inline PTX keeps
// the compiler from turning them into read-only loads.
__device__ __forceinline__ float ld_ca(const float *p) {
    float v;
    asm volatile("ld.global.ca.f32 %0, [%1];" : "=f"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ double ld_ca(const double *p) {
    double v;
    asm volatile("ld.global.ca.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ unsigned ld_ca(const unsigned *p) {
    unsigned v;
    asm volatile("ld.global.ca.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ __half ld_ca(const __half *p) {
    unsigned short v;
    asm volatile("ld.global.ca.b16 %0, [%1];" : "=h"(v) : "l"(p) : "memory");
    return __ushort_as_half(v);
}
__device__ __forceinline__ __nv_bfloat16 ld_ca(const __nv_bfloat16 *p) {
    unsigned short v;
    asm volatile("ld.global.ca.b16 %0, [%1];" : "=h"(v) : "l"(p) : "memory");
    return __ushort_as_bfloat16(v);
}
__device__ __forceinline__ float4 ld_ca(const float4 *p) {
    float4 v;
    asm volatile("ld.global.ca.v4.f32 {%0, %1, %2, %3}, [%4];"
                 : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
                 : "l"(p)
                 : "memory");
    return v;
}
__device__ __forceinline__ double2 ld_ca(const double2 *p) {
    double2 v;
    asm volatile("ld.global.ca.v2.f64 {%0, %1}, [%2];" : "=d"(v.x), "=d"(v.y) : "l"(p) : "memory");
    return v;
}
template <bool kCG, typename T>
__device__ __forceinline__ T ld_ro(const T *p) {
    if constexpr (kCG)
        return ld_ca(p);
    else
        return __ldg(p);
}

// ---- population storage: S is the stored type, arithmetic is float or double ----
// Populations are stored as deviations g_i = f_i - w_i from the resting
// equilibrium; half and bfloat16 storage scale them by kHalfScale to stay
// clear of subnormals.
constexpr float kHalfScale = 256.0f;

template <typename S, typename R>
struct Pop;
template <>
struct Pop<double, double> {
    __device__ static double ld(const double *p) { return __ldg(p); }
    __device__ static void st(double *p, double v) { __stcs(p, v); }
    __device__ static double from(double v) { return v; }
    __device__ static double to(double v) { return v; }
    // raw: the stored value itself (the deviation times 2^kScaleLog2)
    static constexpr int kScaleLog2 = 0;
    __device__ static double ld_raw(const double *p) { return __ldg(p); }
    __device__ static void st_raw(double *p, double v) { __stcs(p, v); }
    __device__ static double from_raw(double v) { return v; }
    __device__ static double to_raw(double v) { return v; }
};
template <>
struct Pop<float, float> {
    __device__ static float ld(const float *p) { return __ldg(p); }
    __device__ static void st(float *p, float v) { __stcs(p, v); }
    __device__ static float from(float v) { return v; }
    __device__ static float to(float v) { return v; }
    static constexpr int kScaleLog2 = 0;
    __device__ static float ld_raw(const float *p) { return __ldg(p); }
    __device__ static void st_raw(float *p, float v) { __stcs(p, v); }
    __device__ static float from_raw(float v) { return v; }
    __device__ static float to_raw(float v) { return v; }
};
template <>
struct Pop<__half, float> {
    __device__ static float ld(const __half *p) { return __half2float(__ldg(p)) * (1.0f / kHalfScale); }
    __device__ static void st(__half *p, float v) { *p = __float2half_rn(v * kHalfScale); }
    __device__ static float from(__half v) { return __half2float(v) * (1.0f / kHalfScale); }
    __device__ static __half to(float v) { return __float2half_rn(v * kHalfScale); }
    static constexpr int kScaleLog2 = 8;  // kHalfScale = 2^8
    __device__ static float ld_raw(const __half *p) { return __half2float(__ldg(p)); }
    __device__ static void st_raw(__half *p, float v) { *p = __float2half_rn(v); }
    __device__ static float from_raw(__half v) { return __half2float(v); }
    __device__ static __half to_raw(float v) { return __float2half_rn(v); }
};
template <>
struct Pop<__nv_bfloat16, float> {
    __device__ static float ld(const __nv_bfloat16 *p) {
        return __bfloat162float(__ldg(p)) * (1.0f / kHalfScale);
    }
    __device__ static void st(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v * kHalfScale); }
    __device__ static float from(__nv_bfloat16 v) { return __bfloat162float(v) * (1.0f / kHalfScale); }
    __device__ static __nv_bfloat16 to(float v) { return __float2bfloat16_rn(v * kHalfScale); }
    // stochastic rounding: adding 16 uniform random bits below the bfloat16
    // mantissa and truncating rounds the magnitude up with probability equal
    // to the discarded fraction, so the stored value is unbiased
    static constexpr int kScaleLog2 = 8;  // kHalfScale = 2^8
    __device__ static float ld_raw(const __nv_bfloat16 *p) { return __bfloat162float(__ldg(p)); }
    __device__ static void st_raw(__nv_bfloat16 *p, float v) { *p = __float2bfloat16_rn(v); }
    __device__ static float from_raw(__nv_bfloat16 v) { return __bfloat162float(v); }
    __device__ static __nv_bfloat16 to_raw(float v) { return __float2bfloat16_rn(v); }
    // r16: 16 random bits added below the kept mantissa before truncation
    __device__ static __nv_bfloat16 to_sr_bits(float v, uint32_t r16) {
        const uint32_t b = (__float_as_uint(v) + r16) & 0xFFFF0000u;
        return __ushort_as_bfloat16((unsigned short)(b >> 16));
    }
    __device__ static void st_sr_bits(__nv_bfloat16 *p, float v, uint32_t r16) { *p = to_sr_bits(v, r16); }
    __device__ static __nv_bfloat16 to_sr_raw(float v, uint32_t r) { return to_sr_bits(v, r >> 16); }
    __device__ static void st_sr_raw(__nv_bfloat16 *p, float v, uint32_t r) { *p = to_sr_raw(v, r); }
    __device__ static __nv_bfloat16 to_sr(float v, uint32_t r) { return to_sr_raw(v * kHalfScale, r); }
    __device__ static void st_sr(__nv_bfloat16 *p, float v, uint32_t r) { *p = to_sr(v, r); }
};

// Random bits for stochastic rounding from a counter: lowbias32 (the
// integer hash of C. Wellons' "Prospecting for Hash Functions", 2018) of the
// cell index and the step's seed starts a Weyl sequence per cell (sr_draw).
__device__ __forceinline__ uint32_t lowbias32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}
// Draw k of a cell: base + k * 0x9E3779B9 (the golden-ratio increment is
// odd, so each 16-bit half of the draws steps through its range without
// repeats); the hashed base makes each draw uniform across cells and steps.
__device__ __forceinline__ uint32_t sr_draw(uint32_t base, int k) { return base + (uint32_t)k * 0x9E3779B9u; }

// ---- views passed by value to kernels ----
// Scalar parameters exist in both precisions so that the FP32 kernels never
// touch the (slow) FP64 pipe for them; pick<R>() selects the copy.
struct Lattice {
    int nx, ny, nz;
    int ntx, nty, ntz;      // tiles per axis
    int ncell;              // nx*ny*nz
    long long stride;       // elements between population planes (ncell padded)
    int off32;              // 1: all 19 planes lie within 2^32 elements of the first
    int bc[3];
    double tau;
    double gext[3];
    double wall_u[6][3];
    double dist2_cut;       // largest |X - x_k|^2 whose MLS weight is non-zero
    int sweep_bx, sweep_by; // block shape of the whole-lattice sweep (0: default)
    int sweep_vec;          // 1: row-tile sweep (shared-memory staging, 128-bit loads/stores) where it applies
    int far_per_sm;         // > 0: the far-field sweep keeps this many blocks per SM (grid-stride)
    // derived, double and float copies
    double omega_d, cF_d, nu_d, gext_d[3], uw_d[27][3];
    float omega_f, cF_f, nu_f, gext_f[3], uw_f[27][3], dist2_cut_f;
    // odd (momentum) coefficients 3 w_i omega of the collision for the axis
    // and the diagonal directions, chosen in each precision so that
    // 2 c_ax + 8 c_dg = omega holds exactly: the odd parts then return the
    // momentum they are given without a bias from rounded weights
    double codd_d[2];
    float codd_f[2];
};

template <typename R>
__device__ __forceinline__ R pick(double d, float f);
template <>
__device__ __forceinline__ double pick<double>(double d, float) { return d; }
template <>
__device__ __forceinline__ float pick<float>(double, float f) { return f; }

// Image of coordinate c in [0, n) on a periodic axis (no division when c
// is already inside).
__device__ __forceinline__ int wrap_periodic(int c, int n) {
    if ((unsigned)c < (unsigned)n) return c;
    c %= n;
    return c < 0 ? c + n : c;
}

// Wall velocity table index of a node: per axis 0 (interior), 1 (index-0
// face), 2 (last face); entry = mean velocity of the faces present.
__host__ __device__ constexpr int wall_code(int cx, int cy, int cz) { return cx + 3 * cy + 9 * cz; }

struct BodyView {
    int nv, nt, rigid;
    const double *X;        // [3nv] positions of level n
    const double *Xprev;    // [3nv] positions of level n-1
    double *Xnew;           // [3nv] positions of level n+1 (written)
    const void *Xrel;       // [3nv] R: X - origin of level n
    void *Xrel_next;        // [3nv] R: X - origin of level n+1 (written)
    // [3nv] FP32 membranes: (X - origin) - Xrel, the residual of the rounding
    // to FP32, of level n and n+1 (written); null otherwise
    const float *Xlo;
    float *Xlo_next;
    double *U;              // [3nv] interpolated fluid velocity
    double *Ub;             // [3nv] boundary velocity imposed by the IB force
    double *Fl;             // [3nv] Lagrangian IB force
    // IB markers: the nv vertices, or (centroid) the nt triangle centroids
    int centroid;
    int nm;                 // number of markers: nv or nt
    double *Uc;             // centroid markers [3nt]: interpolated fluid velocity
    double *Flc;            // centroid markers [3nt]: Lagrangian IB force
    void *phi;              // [27nm] R: MLS transfer weights of level n
    int *node;              // [27nm] support node indices
    const int *perm;        // [nm + 2nt] MLS points in cell order (markers, probes), or nullptr
    const int *tri;         // [3nt]
    void *tri_geo;          // [8nt] R: unit normal (3), area, centroid - origin (3), unused
    double *tri_vol;        // [nt] volume terms (x_0 - o) . (e1 x e2)
    void *probe;            // [8nt] R per side: pressure - 1/3, traction tau.n (3)
    // membrane topology (CSR over vertices)
    const int *vh_ptr;      // [nv+1]
    const int *vh_list;     // hinge*4 + role
    const int4 *vh_verts;   // per entry: the hinge's vertices (a, b, c, d)
    const void *vh_par;     // per entry, R: k_s, l0, k_b, theta0 of the hinge
    const int *vt_ptr;      // [nv+1]
    const int *vt_list;     // triangle*3 + corner
    const int4 *hinge;      // (a, b, c, d)
    const void *ks, *l0, *kb, *theta0;  // R per hinge
    double V0, mv, kv;
    double inv_mv, inv_6V0; // 1/m_v, 1/(6 V0)
    double origin[3];       // reference point of relative positions and of the volume sum
    int bend_variant;
    int kinematic;          // membrane markers advected with the fluid (kinematic IB)
    int rigid_force;        // rigid: 0 probe stress jump, 1 momentum exchange
    // rigid body
    const double *Xbody;    // [3nv] rest coordinates about the centre
    double *rstate;         // rigid state block, see RigidState
    // support region: node box of level n (read) and of level n+1 (built)
    const int *bbox;        // [6]: lo xyz, hi xyz (inclusive node coordinates)
    int *bbox_next;         // [6], reset by the moments kernel, filled by the update kernel
    double *vol_part;       // [one per MLS block] partial sums of the volume terms
    int nvol_part;
    unsigned int *vol_count; // blocks of the MLS kernel done (reset by the last one)
    double *vol_sum;        // enclosed volume times 6, written by the last MLS block
    int *err;               // device error word of the context (first error wins)
};

// Device error codes (the values of include/lbib.h).
constexpr int kErrDiverged = -4;   // LBIB_EDIVERGED
constexpr int kErrBodyWall = -5;   // LBIB_EBODY_WALL
constexpr int kErrTimeout = -6;    // LBIB_ETIMEOUT
// A marker moving farther than this in one step (lattice units; dt = 1) has
// left the scheme's range: lattice Boltzmann velocities stay well below the
// speed of sound c_s = 0.577, and the MLS support assumes sub-cell motion.
constexpr double kMaxMarkerStep = 1.0;
// Marker coordinates beyond this magnitude (or non-finite) count as
// diverged; the bound keeps node arithmetic far inside int range.
constexpr double kMaxMarkerCoord = 1e9;

// ---- batches: the lattices of several contexts advanced by common launches ----
// Buffers of one lattice in one phase of the six-step rotation.
struct LatRef {
    const void *fin;
    void *fout, *force, *fields, *mom;
    uint32_t *stamp;   // tile flags of the IB force, nullptr without bodies
    uint32_t *d_step;  // device step counter
    int *err;          // device error word
    uint32_t *sr;      // two-word rounding-seed counter
    int parity;        // parity of the step in this phase
};
// A body in one phase, with the lattice it lives in.
struct BodyRef {
    BodyView v;
    int lat;
    int inc_step;  // the first body of its lattice advances the step counter
};
// Launch tables (device pointers).  The blocks of a batch launch are split
// over its items by prefix sums of per-item block counts; *_blk maps each
// block to its item directly (one cached load instead of a search).
struct BatchTables {
    int nl, nb, nmemb, nrigid, ncen;
    const Lattice *lat;    // [nl]
    const LatRef *ref;     // [6 nl]: phase-major
    const BodyRef *body;   // [6 nb]: phase-major
    const int *sweep_lat;  // [nl] lattice of each sweep slot (launch order)
    const int *sweep_pre;  // [nl + 1] sweep blocks, by slot
    const int *mom_pre;    // [nb + 1] moments blocks
    const int *mls_pre;    // [nb + 1] MLS blocks
    const int *memb_id;    // [nmemb] membrane bodies
    const int *memb_pre;   // [nmemb + 1] blocks of 8 vertex warps
    const int *rigid_id;   // [nrigid] rigid bodies
    const int *rf_pre;     // [nrigid + 1] triangle blocks of the force reduction
    const int *rm_pre;     // [nrigid + 1] blocks of 8 marker warps
    const int *cen_id;     // [ncen] bodies with centroid markers
    const int *cen_pre;    // [ncen + 1] blocks of 8 triangle warps
    const int *sweep_blk, *mom_blk, *mls_blk, *memb_blk, *rf_blk, *rm_blk, *cen_blk;  // item of each block
    int sweep_threads;     // threads per sweep block
    int sweep_cpt;         // cells per sweep thread (blocks per lattice = cells / (threads * cpt))
    int sweep_off32;       // 1: every lattice of the batch has off32 set
};

// ---- persistent batched step: one launch runs several steps of every
// lattice of a batch as a queue of work items ----
// Item kinds in their order within a step.  Every item waits only for
// items of earlier kinds of its own step, or of earlier steps, of its own
// lattice, and the queue holds those earlier: items are taken in ticket
// order, so whatever an item waits for was taken earlier by a running
// block, and the queue cannot deadlock.
enum PKind { kPMom = 0, kPMls, kPMemb, kPRf, kPRm, kPCen, kPSweep, kPKinds };
struct PersistTables {
    int nitems;              // items of the launch (all its steps)
    int nsteps;              // steps per launch
    int phase0;              // rotation phase of the launch's first step
    int sweep_cells;         // lattice cells per sweep item
    long long wait_ns;       // bound on each dependency wait (ns)
    const int4 *items;       // [nitems] in queue order: kind | step << 8, body (IB kinds) or lattice
                             // (sweep), virtual block, block count
    const int *body_lat;     // [nb]: lattice of each body
    const unsigned *need;    // [nl * kPKinds]: items of each kind per step and lattice
    unsigned *ticket;        // next ticket (zero at launch)
    unsigned *abort;         // nonzero once a wait has expired (zero at launch)
    unsigned *done;          // [nl * kPKinds]: items finished in this launch (zero at launch)
};

// Copies a table entry into shared memory with the whole block (the batch
// kernels then read lattice and body parameters at shared-memory latency
// instead of chasing them through global memory).  Ends with a barrier.
template <typename T>
__device__ __forceinline__ void stage_shared(T &dst, const T *src) {
    static_assert(sizeof(T) % 4 == 0, "word copy");
    const uint32_t *s = reinterpret_cast<const uint32_t *>(src);
    uint32_t *d = reinterpret_cast<uint32_t *>(&dst);
    for (int w = threadIdx.x; w < (int)(sizeof(T) / 4); w += blockDim.x) d[w] = __ldg(s + w);
    __syncthreads();
}

// Layout of the rigid-body state block (doubles).
struct RigidState {
    enum {
        XC = 0, Q4 = 3, U = 7, UP = 10, W = 13, WP = 16, XC_OLD = 19, ROT = 22, IB = 31, MASS = 40,
        VOL = 41, DENS = 42, GRAV = 43, IBINV = 46, INVM = 55, SIZE = 56
    };
};

}  // namespace lbib
