// Node-level pieces of the fused stream + wall + collide sweep (Sec. 2.1,
// Eq. evoleq with the equilibrium of Eq. eqfunc and the Guo term of
// Eq. forcing; Zou-He walls): shared by the sweep kernels (sweep.cu) and the
// persistent batched step (ib.cu), which runs them beside the IB phases.
#pragma once

#include <type_traits>

#include "lbib_device.cuh"

namespace lbib {

// representatives of the 9 pairs (i, opp(i)) with i < opp(i)
__host__ __device__ constexpr int pair_rep(int k) {
    return k == 0 ? 1 : k == 1 ? 3 : k == 2 ? 5 : k == 3 ? 7 : k == 4 ? 8 : k == 5 ? 9 : k == 6 ? 10 : k == 7 ? 15 : 16;
}

__host__ __device__ constexpr unsigned dirmask(int a, int sgn) {
    unsigned m = 0;
    for (int i = 0; i < Q; ++i)
        if (ecomp(i, a) * sgn > 0) m |= 1u << i;
    return m;
}

// Zou-He known-velocity wall on a face node with inward normal s*e_A
// (s = +1 on the index-0 face).  In deviation form, with
// sum_{e_A=0} w + 2 sum_{s e_A<0} w = 1:
//   rho = (1 + sum0 g + 2 sumout g) / (1 - s uw_A)
//   N_b = 1/2 sum_{e_A=0} g e_b - rho uw_b / 3
//   g_i = g_opp + 6 w_i rho (e_i . uw) - sum_{b != A} e_ib N_b   (s e_iA > 0)
template <int A, typename R>
__device__ __forceinline__ void zouhe_face(R (&g)[Q], int s, const R *uw) {
    R sum0 = R(0), sumout = R(0), t[3] = {R(0), R(0), R(0)};
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int ea = ecomp(i, A);
        if (ea == 0) {
            sum0 += g[i];
            if (ex(i)) t[0] += R(ex(i)) * g[i];
            if (ey(i)) t[1] += R(ey(i)) * g[i];
            if (ez(i)) t[2] += R(ez(i)) * g[i];
        } else if (s * ea < 0) {
            sumout += g[i];
        }
    }
    const R rho = (R(1) + sum0 + R(2) * sumout) / (R(1) - R(s) * uw[A]);
    R N[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) N[b] = (b == A) ? R(0) : R(0.5) * t[b] - rho * uw[b] / R(3);
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int ea = ecomp(i, A);
        if (ea != 0 && s * ea > 0) {
            const R eu = R(ex(i)) * uw[0] + R(ey(i)) * uw[1] + R(ez(i)) * uw[2];
            R corr = R(0);
#pragma unroll
            for (int b = 0; b < 3; ++b)
                if (b != A && ecomp(i, b) != 0) corr += R(ecomp(i, b)) * N[b];
            g[i] = g[opp(i)] + R(6) * wq<R>(i) * rho * eu - corr;
        }
    }
}

// Edge and corner nodes: unknown populations (incoming through any of the
// node's walls) bounce back with the moving-wall momentum term at the mean
// wall velocity and rho0 = 1; buried links (opposite also unknown) take
// the equilibrium f^eq(1, uw).
template <typename R>
__device__ __forceinline__ void wall_corner(R (&g)[Q], unsigned unknown, const R *uw) {
    const R uu = uw[0] * uw[0] + uw[1] * uw[1] + uw[2] * uw[2];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        if (!((unknown >> i) & 1u)) continue;
        const R eu = R(ex(i)) * uw[0] + R(ey(i)) * uw[1] + R(ez(i)) * uw[2];
        if (!((unknown >> opp(i)) & 1u))
            g[i] = g[opp(i)] + R(6) * wq<R>(i) * eu;
        else
            g[i] = wq<R>(i) * (R(3) * eu + R(4.5) * eu * eu - R(1.5) * uu);
    }
}

// Walls, moments, body force and BGK/Guo collision of node (x, y, z) whose
// streamed populations are g (Eqs. evoleq, eqfunc, forcing; Zou-He walls);
// on return g holds the post-collision populations and rho, u the moments
// of the collision (stored as the macroscopic fields).  g is in stored
// units, the deviations times 2^kLog2S (16-bit storage scales them by 2^8):
// scaling by a power of two commutes with every rounding, so the update runs
// on the scaled values (the four moments and the equilibrium weights carry
// the factor) and gives exactly the scaled result.
template <typename R, int kLog2S = 0, bool kCG = false>
__device__ __forceinline__ void collide_node(R (&g)[Q], R *__restrict__ force, const uint32_t *__restrict__ stamp,
                                             uint32_t step, const Lattice &L, int x, int y, int z, long long idx,
                                             R &rho_o, R &ux_o, R &uy_o, R &uz_o) {
    constexpr R kS = R(1 << kLog2S), kInvS = R(1) / R(1 << kLog2S);  // exact powers of two
    const int nx = L.nx, ny = L.ny, nz = L.nz;
    const long long st = L.stride;
    // walls (faces -x,+x,-y,+y,-z,+z; the index-0 face has inward normal +)
    int nf = 0, fa = 0, fs = 0, code[3] = {0, 0, 0};
    unsigned unknown = 0;
    const int c[3] = {x, y, z}, n[3] = {nx, ny, nz};
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        if (L.bc[a] != kWall) continue;
        int s = 0;
        if (c[a] == 0)
            s = 1;
        else if (c[a] == n[a] - 1)
            s = -1;
        if (!s) continue;
        ++nf;
        fa = a;
        fs = s;
        code[a] = s > 0 ? 1 : 2;
        unknown |= (a == 0 ? (s > 0 ? dirmask(0, 1) : dirmask(0, -1))
                           : a == 1 ? (s > 0 ? dirmask(1, 1) : dirmask(1, -1))
                                    : (s > 0 ? dirmask(2, 1) : dirmask(2, -1)));
    }
    if (nf) {
        if (kLog2S)
#pragma unroll
            for (int i = 0; i < Q; ++i) g[i] *= kInvS;
        const int wc = wall_code(code[0], code[1], code[2]);
        R uw[3];
        for (int b = 0; b < 3; ++b) uw[b] = pick<R>(L.uw_d[wc][b], L.uw_f[wc][b]);
        if (nf == 1) {
            if (fa == 0)
                zouhe_face<0>(g, fs, uw);
            else if (fa == 1)
                zouhe_face<1>(g, fs, uw);
            else
                zouhe_face<2>(g, fs, uw);
        } else {
            wall_corner(g, unknown, uw);
        }
        if (kLog2S)
#pragma unroll
            for (int i = 0; i < Q; ++i) g[i] *= kS;
    }

    // moments of the streamed populations, over the pairs (i, opp(i))
    R dr = g[0], jx = R(0), jy = R(0), jz = R(0);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const int i = pair_rep(k), o = opp(i);
        const R sum = g[i] + g[o], dif = g[i] - g[o];
        dr += sum;
        if (ex(i)) jx += R(ex(i)) * dif;
        if (ey(i)) jy += R(ey(i)) * dif;
        if (ez(i)) jz += R(ez(i)) * dif;
    }
    if (kLog2S) {
        dr *= kInvS;
        jx *= kInvS;
        jy *= kInvS;
        jz *= kInvS;
    }
    const R rho = R(1) + dr;

    // body force f_lb = g_ext + f_ib (none on wall nodes); consume the IB
    // force of flagged tiles
    R F0 = R(0), F1 = R(0), F2 = R(0);
    if (nf == 0) {
        F0 = pick<R>(L.gext_d[0], L.gext_f[0]);
        F1 = pick<R>(L.gext_d[1], L.gext_f[1]);
        F2 = pick<R>(L.gext_d[2], L.gext_f[2]);
    }
    const int tile = (x >> 3) + L.ntx * ((y >> 3) + L.nty * (z >> 3));
    if (stamp && ld_ro<kCG>(stamp + tile) == step) {
        const R fx = force[idx], fy = force[st + idx], fz = force[2 * st + idx];
        force[idx] = R(0);
        force[st + idx] = R(0);
        force[2 * st + idx] = R(0);
        if (nf == 0) {
            F0 += fx;
            F1 += fy;
            F2 += fz;
        }
    }

    // BGK collision with the Guo term, u = (sum f e + f_lb/2)/rho = j'/rho.
    // Per direction, with b = 4.5 omega rho, c3 = 3 cF, c9 = 9 cF and
    // A0 = omega (drho - 1.5 rho u.u) - 3 cF u.F:
    //   g*_i = (1 - omega) g_i + w_i [A0 + E_i] + c_i e.j' + w_i c3 eF,
    //   E_i = eu (b eu + c9 eF) (even in e_i), c_i = 3 w_i omega,
    // which is g - omega (g - (f^eq - w)) + F_i of Eqs. (evoleq, eqfunc,
    // forcing) regrouped so that each pair (i, opp(i)) shares the even and
    // the odd part.  The odd part takes the momentum j' itself (not rho
    // times the rounded u) and coefficients c_i whose momentum sums to
    // omega exactly (L.codd): the rounding of u or of the weights would
    // otherwise shift the momentum the collision returns by the same
    // relative amount step after step in a slowly changing flow, which acts
    // like a small body force.
    const R inv = R(1) / rho;
    const R omega = pick<R>(L.omega_d, L.omega_f);
    const R om1 = R(1) - omega, cb = R(4.5) * omega * rho;
    const R cax = pick<R>(L.codd_d[0], L.codd_f[0]) * kS, cdg = pick<R>(L.codd_d[1], L.codd_f[1]) * kS;
    if (F0 == R(0) && F1 == R(0) && F2 == R(0)) {
        // no body force on this node (the common case): the same update with
        // the Guo terms, which vanish exactly, left out
        const R ux = jx * inv, uy = jy * inv, uz = jz * inv;
        const R uu = ux * ux + uy * uy + uz * uz;
        const R A0 = omega * (dr - R(1.5) * rho * uu);
        g[0] = om1 * g[0] + (wq<R>(0) * kS) * A0;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const int i = pair_rep(k), o = opp(i);
            R eu = R(0), ej = R(0);
            if (ex(i)) { eu += R(ex(i)) * ux; ej += R(ex(i)) * jx; }
            if (ey(i)) { eu += R(ey(i)) * uy; ej += R(ey(i)) * jy; }
            if (ez(i)) { eu += R(ez(i)) * uz; ej += R(ez(i)) * jz; }
            const R w = wq<R>(i) * kS;
            const R E = eu * (cb * eu);
            const R base = w * (A0 + E), odd = (i <= 6 ? cax : cdg) * ej;
            const R gi = om1 * g[i] + (base + odd), go = om1 * g[o] + (base - odd);
            g[i] = gi;
            g[o] = go;
        }
        rho_o = rho;
        ux_o = ux;
        uy_o = uy;
        uz_o = uz;
        return;
    }
    const R jx2 = jx + R(0.5) * F0, jy2 = jy + R(0.5) * F1, jz2 = jz + R(0.5) * F2;
    const R ux = jx2 * inv, uy = jy2 * inv, uz = jz2 * inv;
    const R cF = pick<R>(L.cF_d, L.cF_f);
    const R uu = ux * ux + uy * uy + uz * uz;
    const R uF = ux * F0 + uy * F1 + uz * F2;
    const R c3 = R(3) * cF, c9 = R(9) * cF;
    const R A0 = omega * (dr - R(1.5) * rho * uu) - c3 * uF;
    const R g0 = om1 * g[0] + (wq<R>(0) * kS) * A0;
    g[0] = g0;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const int i = pair_rep(k), o = opp(i);
        R eu = R(0), ej = R(0), eF = R(0);
        if (ex(i)) { eu += R(ex(i)) * ux; ej += R(ex(i)) * jx2; eF += R(ex(i)) * F0; }
        if (ey(i)) { eu += R(ey(i)) * uy; ej += R(ey(i)) * jy2; eF += R(ey(i)) * F1; }
        if (ez(i)) { eu += R(ez(i)) * uz; ej += R(ez(i)) * jz2; eF += R(ez(i)) * F2; }
        const R w = wq<R>(i) * kS;
        const R E = eu * (cb * eu + c9 * eF);
        const R base = w * (A0 + E), odd = (i <= 6 ? cax : cdg) * ej + w * (c3 * eF);
        const R gi = om1 * g[i] + (base + odd), go = om1 * g[o] + (base - odd);
        g[i] = gi;
        g[o] = go;
    }
    rho_o = rho;
    ux_o = ux;
    uy_o = uy;
    uz_o = uz;
}

// Element o of population plane i.  With 32-bit plane offsets (every
// element of the 19 planes within 2^32 of the base, L.off32) the address is
// one 32-bit multiply-add and one widening multiply-add; else the offset is
// formed in 64 bits.
template <bool kOff32, typename T>
__device__ __forceinline__ T *plane_ptr(T *base, const Lattice &L, int i, int o) {
    if constexpr (kOff32)
        return base + ((unsigned)i * (unsigned)L.stride + (unsigned)o);
    else
        return base + ((long long)i * L.stride + o);
}

// Stream, walls and collision of node (x, y, z).  kCG: the populations and
// tile flags may have been written by other blocks of the launch (see
// ld_ro).
template <typename S, typename R, bool kOff32, bool kCG = false>
__device__ __forceinline__ void sweep_cell(const S *__restrict__ fin, S *__restrict__ fout, R *__restrict__ force,
                                           const uint32_t *__restrict__ stamp, uint32_t step, const Lattice &L,
                                           R *__restrict__ fields, int x, int y, int z, uint32_t seed) {
    const int nx = L.nx, ny = L.ny, nz = L.nz;
    const int idx = x + nx * (y + ny * z);
    const bool px = L.bc[0] == kPeriodic, py = L.bc[1] == kPeriodic, pz = L.bc[2] == kPeriodic;
    // neighbour coordinates; on walled axes an outside source is clamped to
    // the node itself (its value is unused: the wall rule overwrites it)
    int xm = x - 1, xp = x + 1, ym = y - 1, yp = y + 1, zm = z - 1, zp = z + 1;
    if (xm < 0) xm = px ? nx - 1 : 0;
    if (xp >= nx) xp = px ? 0 : nx - 1;
    if (ym < 0) ym = py ? ny - 1 : 0;
    if (yp >= ny) yp = py ? 0 : ny - 1;
    if (zm < 0) zm = pz ? nz - 1 : 0;
    if (zp >= nz) zp = pz ? 0 : nz - 1;
    const int nxy = nx * ny;
    const int oy_m = ym * nx, oy_0 = y * nx, oy_p = yp * nx;
    const int oz_m = zm * nxy, oz_0 = z * nxy, oz_p = zp * nxy;
    const long long st = L.stride;

    // pull: f_i(x) = f*_i(x - e_i)
    R g[Q];
#pragma unroll
    for (int i = 0; i < Q; ++i) {
        const int sx = ex(i) > 0 ? xm : ex(i) < 0 ? xp : x;
        const int sy = ey(i) > 0 ? oy_m : ey(i) < 0 ? oy_p : oy_0;
        const int sz = ez(i) > 0 ? oz_m : ez(i) < 0 ? oz_p : oz_0;
        g[i] = Pop<S, R>::from_raw(ld_ro<kCG>(plane_ptr<kOff32>(fin, L, i, sx + sy + sz)));
    }

    R rho, ux, uy, uz;
    collide_node<R, Pop<S, R>::kScaleLog2, kCG>(g, force, stamp, step, L, x, y, z, idx, rho, ux, uy, uz);
    // bfloat16 storage rounds stochastically (8-bit mantissa: nearest
    // rounding of a smooth flow repeats the same error at every node of a
    // plane and step, a bias); the other formats round to nearest
    // (one 32-bit draw rounds g0 and then each pair (i, opp(i)): its high
    // 16 bits for i, its low 16 bits for the opposite direction)
    constexpr bool kSR = std::is_same<S, __nv_bfloat16>::value;
    if constexpr (kSR) {
        const uint32_t base = lowbias32((uint32_t)idx * 0x9E3779B9u ^ lowbias32(seed));
        Pop<S, R>::st_sr_bits(plane_ptr<kOff32>(fout, L, 0, idx), g[0], sr_draw(base, 0) >> 16);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const int i = pair_rep(k), o = opp(i);
            const uint32_t rs = sr_draw(base, k + 1);
            Pop<S, R>::st_sr_bits(plane_ptr<kOff32>(fout, L, i, idx), g[i], rs >> 16);
            Pop<S, R>::st_sr_bits(plane_ptr<kOff32>(fout, L, o, idx), g[o], rs & 0xFFFFu);
        }
    } else {
        Pop<S, R>::st_raw(plane_ptr<kOff32>(fout, L, 0, idx), g[0]);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const int i = pair_rep(k), o = opp(i);
            Pop<S, R>::st_raw(plane_ptr<kOff32>(fout, L, i, idx), g[i]);
            Pop<S, R>::st_raw(plane_ptr<kOff32>(fout, L, o, idx), g[o]);
        }
    }
    if (fields) {
        fields[idx] = rho;
        fields[st + idx] = ux;
        fields[2 * st + idx] = uy;
        fields[3 * st + idx] = uz;
    }
}

}  // namespace lbib
