// Fused stream + wall + collide sweep over the whole lattice (Sec. 2.1,
// Eq. evoleq with the equilibrium of Eq. eqfunc and the Guo term of
// Eq. forcing), plus the kernels that initialise and export populations and
// macroscopic fields.
//
// Design: one thread per node, pull streaming f_i(x) = f*_i(x - e_i) from
// structure-of-arrays planes (x fastest, so every population load and store
// of a warp is one contiguous 128-byte run except at the x-wrap), read-only
// loads through the non-coherent path and evict-first stores.  The IB force
// lives in a dense field that is read (and zeroed) only inside tiles flagged
// for the current step, so untouched tiles cost one cached 4-byte flag read.
#include <type_traits>

#include "lbib_device.cuh"
#include "lbib_kernels.h"
#include "sweep_cell.cuh"

namespace lbib {

// Node box of the current step, clamped to the lattice (walled axes) or to
// one period (periodic axes); ext = 0 on an empty box.
__device__ __forceinline__ void clamp_box(const Lattice &L, const int *box, int *lo, int *ext) {
    const int n[3] = {L.nx, L.ny, L.nz};
    for (int a = 0; a < 3; ++a) {
        long long l = box[a], h = box[3 + a];
        if (a == 0 && h >= l && (L.nx & 3) == 0) {
            // whole groups of 8 (or 4) nodes along x, so that the 16-byte
            // vectors of the row-tile sweep (4 FP32 or 8 FP16/BF16 values)
            // never straddle the far-field and box sweeps
            const long long g = (L.nx & 7) == 0 ? 7LL : 3LL;
            l &= ~g;  // down to a multiple of the group (two's complement: also below 0)
            h |= g;   // up to the last node of its group
        }
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
}

__device__ __forceinline__ bool in_box(const Lattice &L, const int *lo, const int *ext, int x, int y, int z) {
    const int c[3] = {x, y, z}, n[3] = {L.nx, L.ny, L.nz};
    // walled axes first (no wrap; most far-field nodes fail one of them)
#pragma unroll
    for (int a = 0; a < 3; ++a)
        if (L.bc[a] != kPeriodic && (unsigned)(c[a] - lo[a]) >= (unsigned)ext[a]) return false;
#pragma unroll
    for (int a = 0; a < 3; ++a)
        if (L.bc[a] == kPeriodic && (unsigned)wrap_periodic(c[a] - lo[a], n[a]) >= (unsigned)ext[a]) return false;
    return true;
}

// Whole lattice (box == nullptr), or every node outside the box.
// sr: the two-word rounding-seed counter of the lattice; a step reads word
// `parity` and advances the other one (parity alternates with the steps).
template <typename S, typename R, bool kOff32>
__global__ void __launch_bounds__(256) k_sweep(const S *__restrict__ fin, S *__restrict__ fout,
                                               R *__restrict__ force, const uint32_t *__restrict__ stamp,
                                               const uint32_t *__restrict__ dstep, Lattice L,
                                               R *__restrict__ fields, const int *__restrict__ box,
                                               uint32_t *__restrict__ sr, int parity) {
    const uint32_t step = stamp ? *dstep : 0u;
    const uint32_t seed = sr[parity];
    if (blockIdx.x == 0 && blockIdx.y == 0 && blockIdx.z == 0 && threadIdx.x == 0 && threadIdx.y == 0)
        sr[parity ^ 1] = seed + 1u;
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y * blockDim.y + threadIdx.y;
    const int z = blockIdx.z;
    if (x >= L.nx || y >= L.ny) return;
    if (box) {
        int lo[3], ext[3];
        clamp_box(L, box, lo, ext);
        if (in_box(L, lo, ext, x, y, z)) return;
    }
    sweep_cell<S, R, kOff32>(fin, fout, force, stamp, step, L, fields, x, y, z, seed);
}

// The far field (nodes outside the body box) with a bounded number of
// resident blocks: each block strides over the (x-tile, y-tile, z) tiles of
// the lattice, so that SM resources stay free for the IB kernels running
// beside it (the block scheduler cannot take resources back from blocks
// already resident).
template <typename S, typename R, bool kOff32>
__global__ void __launch_bounds__(256) k_sweep_far(const S *__restrict__ fin, S *__restrict__ fout,
                                                   R *__restrict__ force, const uint32_t *__restrict__ stamp,
                                                   const uint32_t *__restrict__ dstep, Lattice L,
                                                   R *__restrict__ fields, const int *__restrict__ box,
                                                   uint32_t *__restrict__ sr, int parity, int gx, int gy) {
    const uint32_t step = stamp ? *dstep : 0u;
    const uint32_t seed = sr[parity];
    if (blockIdx.x == 0 && threadIdx.x == 0 && threadIdx.y == 0) sr[parity ^ 1] = seed + 1u;
    int lo[3], ext[3];
    clamp_box(L, box, lo, ext);
    const int ntile = gx * gy * L.nz;
    for (int t = blockIdx.x; t < ntile; t += gridDim.x) {
        const int tx = t % gx, ty = (t / gx) % gy, z = t / (gx * gy);
        const int x = tx * blockDim.x + threadIdx.x, y = ty * blockDim.y + threadIdx.y;
        if (x >= L.nx || y >= L.ny || in_box(L, lo, ext, x, y, z)) continue;
        sweep_cell<S, R, kOff32>(fin, fout, force, stamp, step, L, fields, x, y, z, seed);
    }
}

// Row-tile sweep with shared-memory staging: a block takes `rows`
// consecutive x-rows of one z-plane.  It first copies, for every direction
// i, the source rows (y - e_iy, z - e_iz) into shared memory with 128-bit
// coalesced loads; each thread then pulls its node's 19 values from shared
// memory (the x shift and its periodic or walled wrap stay inside the row),
// collides, writes the results back over the staged rows, and the block
// stores them with 128-bit coalesced stores.  Needs rows of whole 16-byte
// vectors (nx * sizeof(S) a multiple of 16); with a body box, the box holds
// whole groups of 4 nodes along x, so no vector straddles it.
template <typename S, typename R>
__global__ void __launch_bounds__(512) k_sweep_tile(const S *__restrict__ fin, S *__restrict__ fout,
                                                     R *__restrict__ force, const uint32_t *__restrict__ stamp,
                                                     const uint32_t *__restrict__ dstep, Lattice L,
                                                     R *__restrict__ fields, const int *__restrict__ box,
                                                     uint32_t *__restrict__ sr, int parity, int rows) {
    extern __shared__ uint4 tile_raw[];
    S *sm = reinterpret_cast<S *>(tile_raw);  // [Q][rows][nx]
    constexpr int V = 16 / sizeof(S);         // nodes per 16-byte vector
    const uint32_t step = stamp ? *dstep : 0u;
    const uint32_t seed = sr[parity];
    if (blockIdx.x == 0 && blockIdx.y == 0 && threadIdx.x == 0) sr[parity ^ 1] = seed + 1u;
    const int nx = L.nx, ny = L.ny, nz = L.nz, nxy = nx * ny;
    const int z = blockIdx.y, y0 = blockIdx.x * rows;
    const int nrows = min(rows, ny - y0);
    const int nvec = nx / V;  // vectors per row
    const long long st = L.stride;
    const bool px = L.bc[0] == kPeriodic, py = L.bc[1] == kPeriodic, pz = L.bc[2] == kPeriodic;
    int lo[3] = {0, 0, 0}, ext[3] = {0, 0, 0};
    if (box) clamp_box(L, box, lo, ext);

    // stage the source rows: a thread keeps one (row, vector) slot and
    // takes every G-th direction, so no division sits in the loops
    const int nslot = nrows * nvec, G = blockDim.x / nslot;  // blockDim >= nslot: rows * nx >= rows * nvec
    const int slot = threadIdx.x % nslot, grp = threadIdx.x / nslot;
    const int sr_ = slot / nvec, sq = slot - sr_ * nvec;
    if (grp < G) {
        const int yr = y0 + sr_;
        int ym = yr - 1, yp = yr + 1, zm = z - 1, zp = z + 1;
        if (ym < 0) ym = py ? ny - 1 : 0;
        if (yp >= ny) yp = py ? 0 : ny - 1;
        if (zm < 0) zm = pz ? nz - 1 : 0;
        if (zp >= nz) zp = pz ? 0 : nz - 1;
        for (int i = grp; i < Q; i += G) {
            const int eyi = ey(i), ezi = ez(i);
            const int sy = eyi > 0 ? ym : eyi < 0 ? yp : yr;
            const int sz = ezi > 0 ? zm : ezi < 0 ? zp : z;
            const S *src = fin + (long long)i * st + ((long long)sy * nx + (long long)sz * nxy) + sq * V;
            reinterpret_cast<uint4 *>(sm + (i * rows + sr_) * nx)[sq] = __ldg(reinterpret_cast<const uint4 *>(src));
        }
    }
    __syncthreads();

    const int r = threadIdx.x / nx, x = threadIdx.x - r * nx, y = y0 + r;
    const bool mine = r < nrows && !(box && in_box(L, lo, ext, x, y, z));
    R g[Q];
    if (mine) {
        int xm = x - 1, xp = x + 1;
        if (xm < 0) xm = px ? nx - 1 : 0;
        if (xp >= nx) xp = px ? 0 : nx - 1;
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const int sx = ex(i) > 0 ? xm : ex(i) < 0 ? xp : x;
            g[i] = Pop<S, R>::from_raw(sm[(i * rows + r) * nx + sx]);
        }
        const long long idx = x + (long long)y * nx + (long long)z * nxy;
        R rho, ux, uy, uz;
        collide_node<R, Pop<S, R>::kScaleLog2>(g, force, stamp, step, L, x, y, z, idx, rho, ux, uy, uz);
        if (fields) {
            fields[idx] = rho;
            fields[st + idx] = ux;
            fields[2 * st + idx] = uy;
            fields[3 * st + idx] = uz;
        }
    }
    __syncthreads();  // every staged value has been read
    if (mine) {
        // the rounding of the one-node sweep: bfloat16 rounds stochastically
        // with the cell's random stream, the values taken in the same order
        constexpr bool kSR = std::is_same<S, __nv_bfloat16>::value;
        const long long idx = x + (long long)y * nx + (long long)z * nxy;
        S *row = sm + r * nx + x;  // value of direction i at row[i * rows * nx]
        if constexpr (kSR) {
            const uint32_t base = lowbias32((uint32_t)idx * 0x9E3779B9u ^ lowbias32(seed));
            row[0] = Pop<S, R>::to_sr_bits(g[0], sr_draw(base, 0) >> 16);
#pragma unroll
            for (int k = 0; k < 9; ++k) {
                const int i = pair_rep(k), o = opp(i);
                const uint32_t rs = sr_draw(base, k + 1);
                row[i * rows * nx] = Pop<S, R>::to_sr_bits(g[i], rs >> 16);
                row[o * rows * nx] = Pop<S, R>::to_sr_bits(g[o], rs & 0xFFFFu);
            }
        } else {
#pragma unroll
            for (int i = 0; i < Q; ++i) row[i * rows * nx] = Pop<S, R>::to_raw(g[i]);
        }
    }
    __syncthreads();
    if (grp < G && !(box && in_box(L, lo, ext, sq * V, y0 + sr_, z))) {  // not the box sweep's nodes
        S *dst = fout + ((long long)(y0 + sr_) * nx + (long long)z * nxy) + sq * V;
        for (int i = grp; i < Q; i += G)
            __stcs(reinterpret_cast<uint4 *>(dst + (long long)i * st),
                   reinterpret_cast<const uint4 *>(sm + (i * rows + sr_) * nx)[sq]);
    }
}

// The nodes inside the box (grid-stride; periodic coordinates wrap).
template <typename S, typename R, bool kOff32>
__global__ void __launch_bounds__(256) k_sweep_box(const S *__restrict__ fin, S *__restrict__ fout,
                                                   R *__restrict__ force, const uint32_t *__restrict__ stamp,
                                                   const uint32_t *__restrict__ dstep, Lattice L,
                                                   R *__restrict__ fields, const int *__restrict__ box,
                                                   const uint32_t *__restrict__ sr, int parity) {
    const uint32_t step = stamp ? *dstep : 0u;
    const uint32_t seed = sr[parity];
    int lo[3], ext[3];
    clamp_box(L, box, lo, ext);
    const int total = ext[0] * ext[1] * ext[2];
    const int n[3] = {L.nx, L.ny, L.nz};
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < total; k += gridDim.x * blockDim.x) {
        int c[3] = {lo[0] + k % ext[0], lo[1] + (k / ext[0]) % ext[1], lo[2] + k / (ext[0] * ext[1])};
        for (int a = 0; a < 3; ++a)
            if (L.bc[a] == kPeriodic) c[a] = wrap_periodic(c[a], n[a]);
        sweep_cell<S, R, kOff32>(fin, fout, force, stamp, step, L, fields, c[0], c[1], c[2], seed);
    }
}

// All lattices of a batch: block b belongs to sweep slot sweep_blk[b]; the
// blocks of a lattice stride over its cells (x fastest), a few cells per
// thread so that the per-block set-up (the lattice entry staged in shared
// memory) is amortised.
template <typename S, typename R, bool kOff32>
__global__ void __launch_bounds__(512) kb_sweep(BatchTables T, int phase, int store_fields) {
    __shared__ Lattice L;
    const int slot = __ldg(T.sweep_blk + blockIdx.x);
    const int l = __ldg(T.sweep_lat + slot);
    stage_shared(L, T.lat + l);
    const LatRef &F = T.ref[phase * T.nl + l];
    const int b0 = __ldg(T.sweep_pre + slot), nb = __ldg(T.sweep_pre + slot + 1) - b0;
    const uint32_t step = F.stamp ? *F.d_step : 0u;
    const uint32_t seed = F.sr[F.parity];
    if (blockIdx.x == b0 && threadIdx.x == 0) F.sr[F.parity ^ 1] = seed + 1u;
    R *fields = store_fields ? (R *)F.fields : nullptr;
    for (int c = (blockIdx.x - b0) * blockDim.x + threadIdx.x; c < L.ncell; c += nb * blockDim.x) {
        const int x = c % L.nx, yz = c / L.nx, y = yz % L.ny, z = yz / L.ny;
        sweep_cell<S, R, kOff32>((const S *)F.fin, (S *)F.fout, (R *)F.force, F.stamp, step, L, fields, x, y, z, seed);
    }
}

// f = f^eq(rho, u) from double fields (Eq. eqfunc), stored as deviations.
// rho and u null: density 1 and the linear shear profile u_x = lo + (hi -
// lo) z / (nz - 1) (the fluid at rest for lo = hi = 0).
template <typename S, typename R>
__global__ void k_init_equilibrium(S *__restrict__ fout, Lattice L, const double *__restrict__ rho,
                                   const double *__restrict__ u, R *__restrict__ fields, double lo, double hi) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= L.ncell) return;
    // in the arithmetic precision R; the density excess is formed in double
    // before rounding (rho - 1 is small)
    double sx = 0.0;
    if (!u && L.nz > 1) {
        const int z = idx / (L.nx * L.ny);
        sx = lo + (hi - lo) * z / (double)(L.nz - 1);
    }
    const R dr = rho ? R(rho[idx] - 1.0) : R(0), r = R(1) + dr;
    const R ux = u ? R(u[3 * idx]) : R(sx), uy = u ? R(u[3 * idx + 1]) : R(0), uz = u ? R(u[3 * idx + 2]) : R(0);
    const R uu = ux * ux + uy * uy + uz * uz;
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        R eu = R(0);
        if (ex(i)) eu += R(ex(i)) * ux;
        if (ey(i)) eu += R(ey(i)) * uy;
        if (ez(i)) eu += R(ez(i)) * uz;
        const R w = wq<R>(i);
        const R g = w * dr + w * r * (R(3) * eu + R(4.5) * eu * eu - R(1.5) * uu);
        Pop<S, R>::st(fout + (long long)i * L.stride + idx, g);
    }
    fields[idx] = r;
    fields[L.stride + idx] = ux;
    fields[2 * L.stride + idx] = uy;
    fields[3 * L.stride + idx] = uz;
}

template <typename S, typename R>
__global__ void k_pop_to_aos(const S *__restrict__ fin, Lattice L, double *__restrict__ out) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= L.ncell) return;
#pragma unroll
    for (int i = 0; i < Q; ++i)
        out[(long long)idx * Q + i] = wq<double>(i) + (double)Pop<S, R>::ld(fin + (long long)i * L.stride + idx);
}

template <typename S, typename R>
__global__ void k_aos_to_pop(const double *__restrict__ in, Lattice L, S *__restrict__ fout) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= L.ncell) return;
#pragma unroll
    for (int i = 0; i < Q; ++i)
        Pop<S, R>::st(fout + (long long)i * L.stride + idx, R(in[(long long)idx * Q + i] - wq<double>(i)));
}

template <typename R>
__global__ void k_fields_out(const R *__restrict__ fields, Lattice L, double *__restrict__ rho,
                             double *__restrict__ u) {
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= L.ncell) return;
    if (rho) rho[idx] = (double)fields[idx];
    if (u) {
        u[3 * idx] = (double)fields[L.stride + idx];
        u[3 * idx + 1] = (double)fields[2 * L.stride + idx];
        u[3 * idx + 2] = (double)fields[3 * L.stride + idx];
    }
}

// ---- host-side launchers (one per storage precision) ----
static inline unsigned grid_for(int n, int b) { return (unsigned)((n + b - 1) / b); }

// Block of whole x-rows: bx = nx rounded up to a warp (at most 256), by rows
// so that a block holds about 256 threads; one z-plane per grid layer.
// Row-tile sweep: rows of whole 16-byte vectors, about 256 nodes a block,
// staged rows within kTileSmem bytes.
constexpr int kTileSmem = 160 * 1024;

template <typename S>
static int tile_rows(const Lattice &L) {
    // nx a multiple of 4 also keeps every vector on one side of a body box
    if (!L.sweep_vec || (L.nx & 3) != 0 || (L.nx * (int)sizeof(S)) % 16 != 0 ||
        (L.stride * (long long)sizeof(S)) % 16 != 0)
        return 0;
    int rows = 256 / L.nx;
    if (rows < 1) rows = 1;
    if (rows > L.ny) rows = L.ny;
    if (rows * L.nx > 512) return 0;
    if ((size_t)Q * rows * L.nx * sizeof(S) > (size_t)kTileSmem) return 0;
    return rows;
}

static void sweep_shape(const Lattice &L, dim3 &grid, dim3 &block) {
    int bx = (L.nx + 31) / 32 * 32;
    if (bx > 256) bx = 256;
    int by = 256 / bx;
    if (L.sweep_bx > 0 && L.sweep_by > 0) {  // tuned shape
        bx = L.sweep_bx;
        by = L.sweep_by;
    }
    if (by < 1) by = 1;
    if (by > L.ny) by = L.ny;
    block = dim3(bx, by, 1);
    grid = dim3((L.nx + bx - 1) / bx, (L.ny + by - 1) / by, L.nz);
}

// part: 0 whole lattice, 1 outside the box, 2 inside the box
template <typename S, typename R, bool kOff32>
static cudaError_t sweep_t(const void *fin, void *fout, void *force, const uint32_t *stamp, const uint32_t *step,
                           const Lattice &L, void *fields, int part, const int *box, uint32_t *sr, int parity,
                           int nsm, cudaStream_t s) {
    if (part == 2) {
        k_sweep_box<S, R, kOff32><<<4 * nsm, 256, 0, s>>>((const S *)fin, (S *)fout, (R *)force, stamp, step, L,
                                                  (R *)fields, box, sr, parity);
    } else if (const int rows = tile_rows<S>(L)) {
        const dim3 grid((L.ny + rows - 1) / rows, L.nz);
        const size_t smem = (size_t)Q * rows * L.nx * sizeof(S);
        k_sweep_tile<S, R><<<grid, rows * L.nx, smem, s>>>((const S *)fin, (S *)fout, (R *)force, stamp, step, L,
                                                           (R *)fields, part == 1 ? box : nullptr, sr, parity,
                                                           rows);
    } else if (part == 1 && L.far_per_sm > 0) {
        dim3 grid, block;
        sweep_shape(L, grid, block);
        k_sweep_far<S, R, kOff32><<<L.far_per_sm * nsm, block, 0, s>>>((const S *)fin, (S *)fout, (R *)force, stamp, step,
                                                               L, (R *)fields, box, sr, parity, (int)grid.x,
                                                               (int)grid.y);
    } else {
        dim3 grid, block;
        sweep_shape(L, grid, block);
        k_sweep<S, R, kOff32><<<grid, block, 0, s>>>((const S *)fin, (S *)fout, (R *)force, stamp, step, L, (R *)fields,
                                             part == 1 ? box : nullptr, sr, parity);
    }
    return cudaGetLastError();
}

template <typename S, typename R>
static cudaError_t sweep_any(const void *fin, void *fout, void *force, const uint32_t *stamp, const uint32_t *step,
                             const Lattice &L, void *fields, int part, const int *box, uint32_t *sr, int parity,
                             int nsm, cudaStream_t s) {
    if (L.off32)
        return sweep_t<S, R, true>(fin, fout, force, stamp, step, L, fields, part, box, sr, parity, nsm, s);
    return sweep_t<S, R, false>(fin, fout, force, stamp, step, L, fields, part, box, sr, parity, nsm, s);
}

cudaError_t launch_sweep(int prec, const void *fin, void *fout, void *force, const uint32_t *stamp,
                         const uint32_t *step, const Lattice &L, void *fields, int part, const int *box,
                         uint32_t *sr, int parity, int nsm, cudaStream_t s) {
    switch (prec) {
        case 0: return sweep_any<double, double>(fin, fout, force, stamp, step, L, fields, part, box, sr, parity, nsm, s);
        case 1: return sweep_any<float, float>(fin, fout, force, stamp, step, L, fields, part, box, sr, parity, nsm, s);
        case 2: return sweep_any<__half, float>(fin, fout, force, stamp, step, L, fields, part, box, sr, parity, nsm, s);
        default:
            return sweep_any<__nv_bfloat16, float>(fin, fout, force, stamp, step, L, fields, part, box, sr, parity,
                                                   nsm, s);
    }
}

template <typename S, typename R>
static cudaError_t batch_sweep_t(const BatchTables &T, const BatchGrid &G, int phase, int store, cudaStream_t s) {
    if (G.sweep > 0) {
        if (T.sweep_off32)
            kb_sweep<S, R, true><<<G.sweep, T.sweep_threads, 0, s>>>(T, phase, store);
        else
            kb_sweep<S, R, false><<<G.sweep, T.sweep_threads, 0, s>>>(T, phase, store);
    }
    return cudaGetLastError();
}

cudaError_t launch_batch_sweep(int prec, const BatchTables &T, const BatchGrid &G, int phase, int store_fields,
                               cudaStream_t s) {
    switch (prec) {
        case 0: return batch_sweep_t<double, double>(T, G, phase, store_fields, s);
        case 1: return batch_sweep_t<float, float>(T, G, phase, store_fields, s);
        case 2: return batch_sweep_t<__half, float>(T, G, phase, store_fields, s);
        default: return batch_sweep_t<__nv_bfloat16, float>(T, G, phase, store_fields, s);
    }
}

// Global mass and momentum of the populations in FP64: sum over nodes of
// sum_i f_i and sum_i f_i e_i.  Each node's 19 deviations are summed in the
// arithmetic precision, the nodes in FP64 (the resting weights add 1 per node
// to the mass and nothing to the momentum).  Fixed-order block partials; the
// last block to finish sums them in block order, so the result does not
// depend on scheduling.
constexpr int kTotBlocks = 512;

template <typename S, typename R>
__global__ void __launch_bounds__(256) k_totals(const S *__restrict__ fin, Lattice L, double *__restrict__ part,
                                                unsigned int *__restrict__ count, double *__restrict__ out) {
    __shared__ double red[4][256];
    __shared__ bool last;
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    const long long st = L.stride;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < L.ncell; idx += gridDim.x * blockDim.x) {
        R m = R(0), jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const R gi = Pop<S, R>::ld(fin + (long long)i * st + idx);
            m += gi;
            if (ex(i)) jx += R(ex(i)) * gi;
            if (ey(i)) jy += R(ey(i)) * gi;
            if (ez(i)) jz += R(ez(i)) * gi;
        }
        acc[0] += (double)m;
        acc[1] += (double)jx;
        acc[2] += (double)jy;
        acc[3] += (double)jz;
    }
    for (int q = 0; q < 4; ++q) red[q][threadIdx.x] = acc[q];
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int q = 0; q < 4; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        for (int q = 0; q < 4; ++q) part[4 * blockIdx.x + q] = red[q][0];
        __threadfence();
        last = atomicAdd(count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x < 4) {
        double t = 0.0;
        for (int b = 0; b < (int)gridDim.x; ++b) t += __ldcg(part + 4 * b + threadIdx.x);
        out[threadIdx.x] = threadIdx.x == 0 ? t + (double)L.ncell : t;
    }
    if (threadIdx.x == 0) *count = 0u;
}

template <typename S, typename R>
static cudaError_t totals_t(const void *fin, const Lattice &L, double *part, unsigned int *count, double *out,
                            cudaStream_t s) {
    int g = (L.ncell + 255) / 256;
    if (g > kTotBlocks) g = kTotBlocks;
    k_totals<S, R><<<g, 256, 0, s>>>((const S *)fin, L, part, count, out);
    return cudaGetLastError();
}

cudaError_t launch_totals(int prec, const void *fin, const Lattice &L, double *part, unsigned int *count,
                          double *out, cudaStream_t s) {
    switch (prec) {
        case 0: return totals_t<double, double>(fin, L, part, count, out, s);
        case 1: return totals_t<float, float>(fin, L, part, count, out, s);
        case 2: return totals_t<__half, float>(fin, L, part, count, out, s);
        default: return totals_t<__nv_bfloat16, float>(fin, L, part, count, out, s);
    }
}

int totals_scratch_doubles() { return 4 * kTotBlocks + 8; }

// Divergence watchdog (not part of the method): every node's density must
// be finite and positive and its speed below the lattice speed of sound
// c_s = 1/sqrt(3) (the equilibrium of Eq. eqfunc is a low-Mach expansion: a
// node past c_s has left the range of the scheme), and the total mass, summed
// in FP64 in a fixed order as in k_totals, must stay within tol (relative)
// of the mass of the first check.  A violation sets the error word to
// LBIB_EDIVERGED unless an earlier error holds it.  w[0]: mass of the first
// check (0 until taken), w[1]: mass of the last check; part: 2 doubles per
// block (mass partial, bad-node flag); count starts and ends at zero.
template <typename S, typename R>
__global__ void __launch_bounds__(256) k_watch(const S *__restrict__ fin, Lattice L, double *__restrict__ part,
                                               unsigned int *__restrict__ count, double *__restrict__ w, double tol,
                                               int *__restrict__ err) {
    __shared__ double red[256];
    __shared__ bool last;
    double acc = 0.0;
    bool bad = false;
    const long long st = L.stride;
    for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < L.ncell; idx += gridDim.x * blockDim.x) {
        R m = R(0), jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
        for (int i = 0; i < Q; ++i) {
            const R gi = Pop<S, R>::ld(fin + (long long)i * st + idx);
            m += gi;
            if (ex(i)) jx += R(ex(i)) * gi;
            if (ey(i)) jy += R(ey(i)) * gi;
            if (ez(i)) jz += R(ez(i)) * gi;
        }
        const R rho = R(1) + m;
        // written so that a NaN anywhere makes the test fail
        const bool ok = rho > R(0) && rho < R(1e30) && R(3) * (jx * jx + jy * jy + jz * jz) < rho * rho;
        bad = bad || !ok;
        acc += (double)m;
    }
    bad = __syncthreads_or(bad) != 0;
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int k = blockDim.x / 2; k > 0; k >>= 1) {
        if ((int)threadIdx.x < k) red[threadIdx.x] += red[threadIdx.x + k];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = red[0];
        part[2 * blockIdx.x + 1] = bad ? 1.0 : 0.0;
        __threadfence();
        last = atomicAdd(count, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    if (!last || threadIdx.x != 0) return;
    __threadfence();
    double mass = 0.0, nbad = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) {
        mass += __ldcg(part + 2 * b);
        nbad += __ldcg(part + 2 * b + 1);
    }
    mass += (double)L.ncell;
    const double m0 = w[0];
    bool diverged = nbad > 0.0 || !(fabs(mass) < 1e300);
    if (!diverged && m0 != 0.0) diverged = !(fabs(mass - m0) <= tol * fabs(m0));
    if (!diverged && m0 == 0.0) w[0] = mass;
    w[1] = mass;
    if (diverged) atomicCAS(err, 0, kErrDiverged);
    *count = 0u;
}

template <typename S, typename R>
static cudaError_t watch_t(const void *fin, const Lattice &L, double *part, unsigned int *count, double *w,
                           double tol, int *err, cudaStream_t s) {
    int g = (L.ncell + 255) / 256;
    if (g > kTotBlocks) g = kTotBlocks;
    k_watch<S, R><<<g, 256, 0, s>>>((const S *)fin, L, part, count, w, tol, err);
    return cudaGetLastError();
}

cudaError_t launch_watch(int prec, const void *fin, const Lattice &L, double *part, unsigned int *count, double *w,
                         double tol, int *err, cudaStream_t s) {
    switch (prec) {
        case 0: return watch_t<double, double>(fin, L, part, count, w, tol, err, s);
        case 1: return watch_t<float, float>(fin, L, part, count, w, tol, err, s);
        case 2: return watch_t<__half, float>(fin, L, part, count, w, tol, err, s);
        default: return watch_t<__nv_bfloat16, float>(fin, L, part, count, w, tol, err, s);
    }
}

// Kernel attributes set once before any launch or capture.
cudaError_t prepare_sweep_kernels() {
    cudaError_t e = cudaFuncSetAttribute(k_sweep_tile<float, float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         kTileSmem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_sweep_tile<double, double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 kTileSmem);
    return e;
}

cudaError_t launch_init_equilibrium(int prec, void *fout, const Lattice &L, const double *rho, const double *u,
                                    void *fields, cudaStream_t s, double shear_lo, double shear_hi) {
    const unsigned g = grid_for(L.ncell, 256);
    const double a = shear_lo, b = shear_hi;
    switch (prec) {
        case 0: k_init_equilibrium<double, double><<<g, 256, 0, s>>>((double *)fout, L, rho, u, (double *)fields, a, b); break;
        case 1: k_init_equilibrium<float, float><<<g, 256, 0, s>>>((float *)fout, L, rho, u, (float *)fields, a, b); break;
        case 2: k_init_equilibrium<__half, float><<<g, 256, 0, s>>>((__half *)fout, L, rho, u, (float *)fields, a, b); break;
        default:
            k_init_equilibrium<__nv_bfloat16, float><<<g, 256, 0, s>>>((__nv_bfloat16 *)fout, L, rho, u,
                                                                      (float *)fields, a, b);
    }
    return cudaGetLastError();
}

cudaError_t launch_pop_to_aos(int prec, const void *fin, const Lattice &L, double *out, cudaStream_t s) {
    const unsigned g = grid_for(L.ncell, 256);
    switch (prec) {
        case 0: k_pop_to_aos<double, double><<<g, 256, 0, s>>>((const double *)fin, L, out); break;
        case 1: k_pop_to_aos<float, float><<<g, 256, 0, s>>>((const float *)fin, L, out); break;
        case 2: k_pop_to_aos<__half, float><<<g, 256, 0, s>>>((const __half *)fin, L, out); break;
        default: k_pop_to_aos<__nv_bfloat16, float><<<g, 256, 0, s>>>((const __nv_bfloat16 *)fin, L, out);
    }
    return cudaGetLastError();
}

cudaError_t launch_aos_to_pop(int prec, const double *in, const Lattice &L, void *fout, cudaStream_t s) {
    const unsigned g = grid_for(L.ncell, 256);
    switch (prec) {
        case 0: k_aos_to_pop<double, double><<<g, 256, 0, s>>>(in, L, (double *)fout); break;
        case 1: k_aos_to_pop<float, float><<<g, 256, 0, s>>>(in, L, (float *)fout); break;
        case 2: k_aos_to_pop<__half, float><<<g, 256, 0, s>>>(in, L, (__half *)fout); break;
        default: k_aos_to_pop<__nv_bfloat16, float><<<g, 256, 0, s>>>(in, L, (__nv_bfloat16 *)fout);
    }
    return cudaGetLastError();
}

cudaError_t launch_fields_out(int prec, const void *fields, const Lattice &L, double *rho, double *u,
                              cudaStream_t s) {
    const unsigned g = grid_for(L.ncell, 256);
    if (prec == 0)
        k_fields_out<double><<<g, 256, 0, s>>>((const double *)fields, L, rho, u);
    else
        k_fields_out<float><<<g, 256, 0, s>>>((const float *)fields, L, rho, u);
    return cudaGetLastError();
}

}  // namespace lbib
