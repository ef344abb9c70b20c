/*
 * lbib_oracle.c -- plain, slow, FP64 CPU statement of the lattice-Boltzmann /
 * dynamic-immersed-boundary method of Coclite, Ranaldo, Pascazio and
 * de Tullio, "A Lattice Boltzmann dynamic-Immersed Boundary scheme for the
 * transport of deformable inertial capsules in low-Re flows" (arXiv 2207.06029).
 *
 * TEST INFRASTRUCTURE.  This file exists to check the CUDA library; it is not
 * part of the product.  Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark may load it.  It shares no code, header, table or
 * helper with the CUDA path.  Every floating-point quantity is a double;
 * build with -ffp-contract=off so that each operation rounds as written.
 *
 * Layout of this oracle: f[idx*19 + i], idx = x + nx*(y + ny*z); node (x,y,z)
 * sits at position (x,y,z) in lattice units (dx = dt = 1, rho0 = 1).
 *
 * Readings of the paper taken where it is silent or garbled are marked
 * "reading:" at the place they act.
 *
 * Pins: every exported function is checked by the "not gpu" tests against
 * something other than itself -- the printed lattice, moment identities,
 * conservation laws, brute-force streaming, exact discrete steady states
 * (Couette, Poiseuille interior), closed forms (MLS on a node, pressure jump
 * of a linear density, platonic dihedral angles, cube inertia, Stokes
 * rotation of a free sphere in shear), finite differences of the
 * membrane energies, and, for the IB markers (vertices or, as printed,
 * triangle centroids), the exact first-step displacement of kinematic
 * markers in the discrete Couette state and the momentum total of the
 * spread force.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define Q 19

/* ------------------------------------------------------------------------ */
/* D3Q19 molecule: columns of the matrix in Eq. (e_i), Sec. 2.1.            */
/* ------------------------------------------------------------------------ */
static const int E[Q][3] = {
    {0, 0, 0},  {1, 0, 0},  {-1, 0, 0}, {0, 1, 0},   {0, -1, 0},
    {0, 0, 1},  {0, 0, -1}, {1, 1, 0},  {1, -1, 0},  {1, 0, 1},
    {1, 0, -1}, {-1, 1, 0}, {-1, -1, 0}, {-1, 0, 1}, {-1, 0, -1},
    {0, 1, 1},  {0, 1, -1}, {0, -1, 1}, {0, -1, -1}};

/* weights stated after Eq. (eqfunc): w0 = 1/3, w1-6 = 1/18, w7-18 = 1/36 */
static double weight(int i) {
    if (i == 0) return 1.0 / 3.0;
    if (i <= 6) return 1.0 / 18.0;
    return 1.0 / 36.0;
}

/* reticular sound speed c_s = 1/sqrt(3) (Sec. 2.1) */
static const double CS2 = 1.0 / 3.0;

/* index j with e_j = -e_i, found by search */
static int opposite(int i) {
    for (int j = 0; j < Q; ++j)
        if (E[j][0] == -E[i][0] && E[j][1] == -E[i][1] && E[j][2] == -E[i][2]) return j;
    return -1;
}

enum { ORC_OK = 0, ORC_EINVAL = -1, ORC_ENOMEM = -2, ORC_EBODY_WALL = -5 };
enum { BC_PERIODIC = 0, BC_WALL = 1 };

void orc_lattice(int *e, double *w) {
    for (int i = 0; i < Q; ++i) {
        for (int a = 0; a < 3; ++a) e[3 * i + a] = E[i][a];
        w[i] = weight(i);
    }
}

/* Eq. (eqfunc): second-order Maxwell-Boltzmann projection. */
void orc_feq(double rho, const double *u, double *feq) {
    double uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    for (int i = 0; i < Q; ++i) {
        double eu = E[i][0] * u[0] + E[i][1] * u[1] + E[i][2] * u[2];
        feq[i] = weight(i) * rho *
                 (1.0 + eu / CS2 + (eu * eu) / (2.0 * CS2 * CS2) - uu / (2.0 * CS2));
    }
}

/* Eq. (forcing): Guo projection of the body force f_lb on direction i. */
void orc_guo(const double *u, const double *flb, double tau, double *out) {
    for (int i = 0; i < Q; ++i) {
        double eu = E[i][0] * u[0] + E[i][1] * u[1] + E[i][2] * u[2];
        double s = 0.0;
        for (int a = 0; a < 3; ++a)
            s += ((E[i][a] - u[a]) / CS2 + eu / (CS2 * CS2) * E[i][a]) * flb[a];
        out[i] = (1.0 - 1.0 / (2.0 * tau)) * weight(i) * s;
    }
}

/* Right-hand side of Eq. (evoleq) for one node with dt = 1: moments
 * rho = sum f, rho u = sum f e + f_lb/2 (Sec. 2.1), then BGK relaxation
 * towards f^eq plus the Guo term.  f is replaced by the post-collision
 * populations; rho and u of the collision are returned. */
void orc_collide(double *f, double tau, const double *flb, double *rho_out, double *u_out) {
    double rho = 0.0, m[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < Q; ++i) {
        rho += f[i];
        for (int a = 0; a < 3; ++a) m[a] += f[i] * E[i][a];
    }
    double u[3];
    for (int a = 0; a < 3; ++a) u[a] = (m[a] + 0.5 * flb[a]) / rho;
    double feq[Q], F[Q];
    orc_feq(rho, u, feq);
    orc_guo(u, flb, tau, F);
    for (int i = 0; i < Q; ++i) f[i] = f[i] - (f[i] - feq[i]) / tau + F[i];
    if (rho_out) *rho_out = rho;
    if (u_out)
        for (int a = 0; a < 3; ++a) u_out[a] = u[a];
}

/* Known-velocity wall of Zou and He (Sec. 2.1, cited after Eq. forcing) on a
 * face node.  reading: the D3Q19 form of the scheme (non-equilibrium
 * bounce-back of the unknown populations plus a transverse-momentum
 * correction), with the wall node itself a fluid node.
 *   axis a, inward normal sign s (+1 on the index-0 face, -1 on the last).
 *   Unknown populations are those with s*e_a > 0.  With the wall velocity uw:
 *     rho = (sum_{e_a=0} f + 2 sum_{s e_a<0} f) / (1 - s uw_a)
 *     N_b = 1/2 sum_{e_a=0} f e_b - rho uw_b / 3          (b tangential)
 *     f_i = f_opp(i) + 6 w_i rho (e_i . uw) - sum_b e_ib N_b
 * The unknown entries of f are overwritten; the rest are read only. */
void orc_zouhe_face(double *f, int a, int s, const double *uw) {
    double sum0 = 0.0, sumout = 0.0;
    for (int i = 0; i < Q; ++i) {
        if (E[i][a] == 0)
            sum0 += f[i];
        else if (s * E[i][a] < 0)
            sumout += f[i];
    }
    double rho = (sum0 + 2.0 * sumout) / (1.0 - s * uw[a]);
    double N[3] = {0.0, 0.0, 0.0};
    for (int b = 0; b < 3; ++b) {
        if (b == a) continue;
        double t = 0.0;
        for (int i = 0; i < Q; ++i)
            if (E[i][a] == 0) t += f[i] * E[i][b];
        N[b] = 0.5 * t - rho * uw[b] / 3.0;
    }
    for (int i = 0; i < Q; ++i) {
        if (s * E[i][a] <= 0) continue;
        double eu = E[i][0] * uw[0] + E[i][1] * uw[1] + E[i][2] * uw[2];
        double corr = 0.0;
        for (int b = 0; b < 3; ++b)
            if (b != a) corr += E[i][b] * N[b];
        f[i] = f[opposite(i)] + 6.0 * weight(i) * rho * eu - corr;
    }
}

/* Edge and corner nodes of walled boxes; the paper gives no rule there.
 * reading: the node belongs to every face it lies on, so no fluid may cross
 * any of them: the wall velocity's component along the normal of one of the
 * node's faces is that face's own normal component, and a component along
 * which none of its faces is normal is the mean of the faces' components.
 * (A lid sliding into a resting side wall thus leaves that edge at rest;
 * taking the plain mean there would give the edge a velocity through the
 * side wall, a source and a sink of mass at the two ends of the lid whose
 * strength shrinks only like the spacing.)  The reference density is
 * rho0 = 1.  An unknown population (s_j e_ia_j > 0 for some face j) whose
 * opposite is known is bounced back with the moving-wall momentum term,
 *     f_i = f_opp + 6 w_i rho0 (e_i . uw);
 * one whose opposite is unknown too (a buried link) is set to
 * f^eq_i(rho0, uw). */
void orc_wall_multi(double *f, int nface, const int *axes, const int *signs, const double *uw_faces) {
    double uw[3] = {0.0, 0.0, 0.0};
    for (int a = 0; a < 3; ++a) {
        int normal_face = -1;
        for (int j = 0; j < nface; ++j)
            if (axes[j] == a) normal_face = j;
        if (normal_face >= 0) {
            uw[a] = uw_faces[3 * normal_face + a];
        } else {
            for (int j = 0; j < nface; ++j) uw[a] += uw_faces[3 * j + a] / nface;
        }
    }
    int unknown[Q];
    for (int i = 0; i < Q; ++i) {
        unknown[i] = 0;
        for (int j = 0; j < nface; ++j)
            if (signs[j] * E[i][axes[j]] > 0) unknown[i] = 1;
    }
    double feq[Q];
    orc_feq(1.0, uw, feq);
    double known_val[Q];
    for (int i = 0; i < Q; ++i) known_val[i] = f[i];
    for (int i = 0; i < Q; ++i) {
        if (!unknown[i]) continue;
        int o = opposite(i);
        if (!unknown[o]) {
            double eu = E[i][0] * uw[0] + E[i][1] * uw[1] + E[i][2] * uw[2];
            f[i] = known_val[o] + 6.0 * weight(i) * 1.0 * eu;
        } else {
            f[i] = feq[i];
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Moving-least-squares transfer (Sec. 2.2, Eqs. uLag, l2norm, intKernel).   */
/* ------------------------------------------------------------------------ */
static const double MLS_RW = 1.3;    /* support size r_w = 1.3 dx */
static const double MLS_ALPHA = 0.3; /* alpha in Eq. (intKernel) */

/* Gauss-Jordan inverse of a 4x4 matrix with partial pivoting. */
static int inverse4(const double *A, double *Ainv) {
    double M[4][8];
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 8; ++c) M[r][c] = (c < 4) ? A[4 * r + c] : (c - 4 == r ? 1.0 : 0.0);
    for (int col = 0; col < 4; ++col) {
        int piv = col;
        for (int r = col + 1; r < 4; ++r)
            if (fabs(M[r][col]) > fabs(M[piv][col])) piv = r;
        if (M[piv][col] == 0.0) return -1;
        if (piv != col)
            for (int c = 0; c < 8; ++c) {
                double t = M[col][c];
                M[col][c] = M[piv][c];
                M[piv][c] = t;
            }
        double d = M[col][col];
        for (int c = 0; c < 8; ++c) M[col][c] /= d;
        for (int r = 0; r < 4; ++r) {
            if (r == col) continue;
            double g = M[r][col];
            if (g == 0.0) continue;
            for (int c = 0; c < 8; ++c) M[r][c] -= g * M[col][c];
        }
    }
    for (int r = 0; r < 4; ++r)
        for (int c = 0; c < 4; ++c) Ainv[4 * r + c] = M[r][c + 4];
    return 0;
}

/* MLS shape functions at point X.
 * The 27 Eulerian points are the 3x3x3 block around the nearest node
 * base = floor(X + 1/2) (reading of the "cube of side r_w" that holds 27
 * points), ordered k = (dz+1)*9 + (dy+1)*3 + (dx+1).
 * Weight (Eq. intKernel): r_k = |X - x_k| / r_w, W = exp(-(r_k/alpha)^2) for
 * r_k <= 1, else 0.
 * Linear basis (Eq. l2norm), written in coordinates shifted to X:
 * p_k = (1, x_k - X); reading: this is the same fit as p = (1,x,y,z) and
 * gives U(X) = a_0, grad U(X) = (a_1, a_2, a_3).
 * Minimising J gives A a = sum_k W_k p_k u_k with A = sum_k W_k p_k p_k^T,
 * so a = sum_k psi_k u_k with psi_k = W_k A^{-1} p_k; phi_k = psi_k[0] is the
 * transfer operator of Eq. (uLag).
 * Outputs: base[3], psi[27*4]; node coordinates are base + (dx,dy,dz). */
int orc_mls_point(const double *X, int *base, double *psi) {
    for (int a = 0; a < 3; ++a) base[a] = (int)floor(X[a] + 0.5);
    double A[16] = {0.0}, Wk[27], P[27][4];
    for (int k = 0; k < 27; ++k) {
        int d[3] = {k % 3 - 1, (k / 3) % 3 - 1, k / 9 - 1};
        double dist2 = 0.0;
        P[k][0] = 1.0;
        for (int a = 0; a < 3; ++a) {
            double xa = (double)(base[a] + d[a]) - X[a];
            P[k][a + 1] = xa;
            dist2 += xa * xa;
        }
        double r = sqrt(dist2) / MLS_RW;
        Wk[k] = (r <= 1.0) ? exp(-(r / MLS_ALPHA) * (r / MLS_ALPHA)) : 0.0;
        for (int i = 0; i < 4; ++i)
            for (int j = 0; j < 4; ++j) A[4 * i + j] += Wk[k] * P[k][i] * P[k][j];
    }
    double Ainv[16];
    if (inverse4(A, Ainv)) return ORC_EINVAL;
    for (int k = 0; k < 27; ++k)
        for (int i = 0; i < 4; ++i) {
            double s = 0.0;
            for (int j = 0; j < 4; ++j) s += Ainv[4 * i + j] * P[k][j];
            psi[4 * k + i] = Wk[k] * s;
        }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Membrane network (Sec. 2.3, Eqs. strainPot/strainFor, bendPot/bendFor,    */
/* volFor).                                                                  */
/* ------------------------------------------------------------------------ */
static void sub3(const double *a, const double *b, double *o) {
    for (int i = 0; i < 3; ++i) o[i] = a[i] - b[i];
}
static void cross3(const double *a, const double *b, double *o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static double norm3(const double *a) { return sqrt(dot3(a, a)); }

/* Triangle (i,j,k), counter-clockwise seen from outside: outward normal
 * N = (x_j - x_i) x (x_k - x_i), area |N|/2, centroid (x_i + x_j + x_k)/3. */
static void tri_geom(const double *X, const int *t, double *n_unit, double *area, double *cen) {
    double e1[3], e2[3], N[3];
    sub3(&X[3 * t[1]], &X[3 * t[0]], e1);
    sub3(&X[3 * t[2]], &X[3 * t[0]], e2);
    cross3(e1, e2, N);
    double nn = norm3(N);
    *area = 0.5 * nn;
    for (int a = 0; a < 3; ++a) {
        n_unit[a] = N[a] / nn;
        cen[a] = (X[3 * t[0] + a] + X[3 * t[1] + a] + X[3 * t[2] + a]) / 3.0;
    }
}

/* Enclosed volume of a closed, outward-oriented triangulation:
 * V = 1/6 sum_t x_i . (x_j x x_k). */
double orc_volume(const double *X, int nt, const int *tri) {
    double V = 0.0;
    for (int t = 0; t < nt; ++t) {
        double c[3];
        cross3(&X[3 * tri[3 * t + 1]], &X[3 * tri[3 * t + 2]], c);
        V += dot3(&X[3 * tri[3 * t]], c) / 6.0;
    }
    return V;
}

double orc_area(const double *X, int nt, const int *tri) {
    double A = 0.0;
    for (int t = 0; t < nt; ++t) {
        double n[3], a, c[3];
        tri_geom(X, &tri[3 * t], n, &a, c);
        A += a;
    }
    return A;
}

/* Topology of a closed oriented manifold triangulation: one hinge per
 * undirected edge, (a, b, c, d) with T1 = (a, b, c) and T2 = (b, a, d) the
 * two triangles sharing edge a-b (Fig. IB c).  Returns the number of hinges,
 * or -1 if some directed edge is not matched exactly once by its reverse.
 * hinge_tri (optional) receives the indices of T1 and T2. */
typedef struct {
    int64_t key;
    int tri, third;
} dedge_t;
static int cmp_dedge(const void *p, const void *q) {
    int64_t a = ((const dedge_t *)p)->key, b = ((const dedge_t *)q)->key;
    return (a > b) - (a < b);
}
int orc_mesh_hinges(int nv, int nt, const int *tri, int *hinge, int *hinge_tri) {
    int nd = 3 * nt;
    dedge_t *d = (dedge_t *)malloc(sizeof(dedge_t) * (size_t)nd);
    if (!d) return -1;
    for (int t = 0; t < nt; ++t)
        for (int s = 0; s < 3; ++s) {
            int a = tri[3 * t + s], b = tri[3 * t + (s + 1) % 3], c = tri[3 * t + (s + 2) % 3];
            d[3 * t + s].key = (int64_t)a * nv + b;
            d[3 * t + s].tri = t;
            d[3 * t + s].third = c;
        }
    qsort(d, (size_t)nd, sizeof(dedge_t), cmp_dedge);
    for (int i = 1; i < nd; ++i)
        if (d[i].key == d[i - 1].key) {
            free(d);
            return -1;
        }
    int nh = 0;
    for (int i = 0; i < nd; ++i) {
        int a = (int)(d[i].key / nv), b = (int)(d[i].key % nv);
        /* find the reverse edge b->a */
        int64_t rk = (int64_t)b * nv + a;
        int lo = 0, hi = nd - 1, found = -1;
        while (lo <= hi) {
            int mid = (lo + hi) / 2;
            if (d[mid].key == rk) {
                found = mid;
                break;
            }
            if (d[mid].key < rk)
                lo = mid + 1;
            else
                hi = mid - 1;
        }
        if (found < 0) {
            free(d);
            return -1;
        }
        if (a < b) {
            hinge[4 * nh + 0] = a;
            hinge[4 * nh + 1] = b;
            hinge[4 * nh + 2] = d[i].third;
            hinge[4 * nh + 3] = d[found].third;
            if (hinge_tri) {
                hinge_tri[2 * nh + 0] = d[i].tri;
                hinge_tri[2 * nh + 1] = d[found].tri;
            }
            ++nh;
        }
    }
    free(d);
    return nh;
}

/* Eqs. (strainPot, strainFor): V = 1/2 k (l - l0)^2 per edge, and
 * F_1 = -k (l - l0) r_12 / l, F_2 = -F_1.  Forces are added to F; the
 * energy is returned. */
double orc_spring_forces(const double *X, int ne, const int *edge, const double *ks, const double *l0,
                         double *F) {
    double En = 0.0;
    for (int e = 0; e < ne; ++e) {
        int i = edge[2 * e], j = edge[2 * e + 1];
        double r12[3];
        sub3(&X[3 * i], &X[3 * j], r12);
        double l = norm3(r12);
        double dl = l - l0[e];
        En += 0.5 * ks[e] * dl * dl;
        for (int a = 0; a < 3; ++a) {
            double f1 = -ks[e] * dl * r12[a] / l;
            F[3 * i + a] += f1;
            F[3 * j + a] -= f1;
        }
    }
    return En;
}

/* Signed dihedral angle of hinge (a, b, c, d) and its gradient.
 * e = x_b - x_a, N1 = e x (x_c - x_a) (normal of T1), N2 = (x_d - x_a) x e
 * (normal of T2); theta = atan2((n1 x n2) . e/|e|, n1 . n2), positive where
 * the surface is convex.  The gradient follows from rotating each triangle
 * about the hinge: with heights h1 = |N1|/|e|, h2 = |N2|/|e| and the edge
 * parameters t_c = (x_c - x_a).e/|e|^2, t_d = (x_d - x_a).e/|e|^2,
 *   dtheta/dx_c = -n1/h1,  dtheta/dx_d = -n2/h2,
 *   dtheta/dx_a = (1-t_c) n1/h1 + (1-t_d) n2/h2,
 *   dtheta/dx_b = t_c n1/h1 + t_d n2/h2.
 * grad (optional) receives 12 numbers in the order a, b, c, d. */
double orc_hinge_theta(const double *xa, const double *xb, const double *xc, const double *xd, double *grad) {
    double e[3], ac[3], ad[3], N1[3], N2[3];
    sub3(xb, xa, e);
    sub3(xc, xa, ac);
    sub3(xd, xa, ad);
    cross3(e, ac, N1);
    cross3(ad, e, N2);
    double le = norm3(e), l1 = norm3(N1), l2 = norm3(N2);
    double n1[3], n2[3], c12[3];
    for (int k = 0; k < 3; ++k) {
        n1[k] = N1[k] / l1;
        n2[k] = N2[k] / l2;
    }
    cross3(n1, n2, c12);
    double theta = atan2(dot3(c12, e) / le, dot3(n1, n2));
    if (grad) {
        double h1 = l1 / le, h2 = l2 / le;
        double tc = dot3(ac, e) / (le * le), td = dot3(ad, e) / (le * le);
        for (int k = 0; k < 3; ++k) {
            double g1 = n1[k] / h1, g2 = n2[k] / h2;
            grad[0 + k] = (1.0 - tc) * g1 + (1.0 - td) * g2;
            grad[3 + k] = tc * g1 + td * g2;
            grad[6 + k] = -g1;
            grad[9 + k] = -g2;
        }
    }
    return theta;
}

/* Bending (Eqs. bendPot, bendFor).  reading: the printed four-node forces
 * with beta_b = k_b sin(theta - theta0)/sin(theta) are the gradient of the
 * hinge energy k_b [1 - cos(theta - theta0)]; variant 0 uses that energy,
 * variant 1 the printed quadratic 1/2 k_b (theta - theta0)^2.  Forces are
 * F = -dE/dx, added to F; the energy is returned. */
double orc_bend_forces(const double *X, int nh, const int *hinge, const double *kb, const double *theta0,
                       int variant, double *F) {
    double En = 0.0;
    for (int h = 0; h < nh; ++h) {
        const int *v = &hinge[4 * h];
        double g[12];
        double th = orc_hinge_theta(&X[3 * v[0]], &X[3 * v[1]], &X[3 * v[2]], &X[3 * v[3]], g);
        double dth = th - theta0[h];
        double dEdth;
        if (variant == 0) {
            En += kb[h] * (1.0 - cos(dth));
            dEdth = kb[h] * sin(dth);
        } else {
            En += 0.5 * kb[h] * dth * dth;
            dEdth = kb[h] * dth;
        }
        for (int q = 0; q < 4; ++q)
            for (int k = 0; k < 3; ++k) F[3 * v[q] + k] -= dEdth * g[3 * q + k];
    }
    return En;
}

/* Volume penalty (Eq. volFor) at each element, shared 1/3 per vertex.
 * reading: the restoring sign, F_t = +k_v (1 - V/V0) n_t A_t with n_t the
 * outward normal, which is -grad of E_v = k_v/(2 V0) (V - V0)^2 because
 * dV/dx_v = 1/3 sum_{t at v} A_t n_t on a closed surface.  Added to F;
 * returns E_v. */
double orc_volume_forces(const double *X, int nt, const int *tri, double kv, double V0, double *F) {
    double V = orc_volume(X, nt, tri);
    for (int t = 0; t < nt; ++t) {
        double n[3], A, c[3];
        tri_geom(X, &tri[3 * t], n, &A, c);
        for (int q = 0; q < 3; ++q)
            for (int k = 0; k < 3; ++k) F[3 * tri[3 * t + q] + k] += kv * (1.0 - V / V0) * n[k] * A / 3.0;
    }
    return kv / (2.0 * V0) * (V - V0) * (V - V0);
}

/* Mass properties of the solid bounded by a closed triangulation with unit
 * density: volume, volume centroid, and inertia tensor about the centroid.
 * Each triangle with the origin spans a tetrahedron of signed volume
 * v = x_i.(x_j x x_k)/6 whose second-moment tensor is
 * v/20 (x_i x_i^T + x_j x_j^T + x_k x_k^T + s s^T), s = x_i + x_j + x_k. */
void orc_mass_properties(const double *X, int nt, const int *tri, double *V_out, double *c_out, double *I_out) {
    double V = 0.0, c[3] = {0, 0, 0}, C[9] = {0};
    for (int t = 0; t < nt; ++t) {
        const double *a = &X[3 * tri[3 * t]], *b = &X[3 * tri[3 * t + 1]], *d = &X[3 * tri[3 * t + 2]];
        double bd[3];
        cross3(b, d, bd);
        double v = dot3(a, bd) / 6.0;
        V += v;
        double s[3];
        for (int k = 0; k < 3; ++k) {
            s[k] = a[k] + b[k] + d[k];
            c[k] += v * s[k] / 4.0;
        }
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                C[3 * i + j] += v / 20.0 * (a[i] * a[j] + b[i] * b[j] + d[i] * d[j] + s[i] * s[j]);
    }
    for (int k = 0; k < 3; ++k) c[k] /= V;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) C[3 * i + j] -= V * c[i] * c[j];
    double tr = C[0] + C[4] + C[8];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) I_out[3 * i + j] = (i == j ? tr : 0.0) - C[3 * i + j];
    *V_out = V;
    for (int k = 0; k < 3; ++k) c_out[k] = c[k];
}

/* ------------------------------------------------------------------------ */
/* Rigid-body kinematics helpers (Sec. 2.3, rigid objects).                 */
/* ------------------------------------------------------------------------ */
static void quat_to_R(const double *q, double *R) {
    double w = q[0], x = q[1], y = q[2], z = q[3];
    R[0] = 1 - 2 * (y * y + z * z);
    R[1] = 2 * (x * y - w * z);
    R[2] = 2 * (x * z + w * y);
    R[3] = 2 * (x * y + w * z);
    R[4] = 1 - 2 * (x * x + z * z);
    R[5] = 2 * (y * z - w * x);
    R[6] = 2 * (x * z - w * y);
    R[7] = 2 * (y * z + w * x);
    R[8] = 1 - 2 * (x * x + y * y);
}
static void quat_mul(const double *p, const double *q, double *o) {
    o[0] = p[0] * q[0] - p[1] * q[1] - p[2] * q[2] - p[3] * q[3];
    o[1] = p[0] * q[1] + p[1] * q[0] + p[2] * q[3] - p[3] * q[2];
    o[2] = p[0] * q[2] - p[1] * q[3] + p[2] * q[0] + p[3] * q[1];
    o[3] = p[0] * q[3] + p[1] * q[2] - p[2] * q[1] + p[3] * q[0];
}
static int inverse3(const double *M, double *Mi) {
    double det = M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) +
                 M[2] * (M[3] * M[7] - M[4] * M[6]);
    if (det == 0.0) return -1;
    Mi[0] = (M[4] * M[8] - M[5] * M[7]) / det;
    Mi[1] = (M[2] * M[7] - M[1] * M[8]) / det;
    Mi[2] = (M[1] * M[5] - M[2] * M[4]) / det;
    Mi[3] = (M[5] * M[6] - M[3] * M[8]) / det;
    Mi[4] = (M[0] * M[8] - M[2] * M[6]) / det;
    Mi[5] = (M[2] * M[3] - M[0] * M[5]) / det;
    Mi[6] = (M[3] * M[7] - M[4] * M[6]) / det;
    Mi[7] = (M[1] * M[6] - M[0] * M[7]) / det;
    Mi[8] = (M[0] * M[4] - M[1] * M[3]) / det;
    return 0;
}

/* Eqs. (linearVelRig, angularVelRig): second-order backward update
 * v(t) = 2/3 (2 v(t-dt) - 1/2 v(t-2dt) + vdot(t) dt), dt = 1. */
void orc_bdf2(const double *v1, const double *v2, const double *vdot, double *out) {
    for (int k = 0; k < 3; ++k) out[k] = 2.0 / 3.0 * (2.0 * v1[k] - 0.5 * v2[k] + vdot[k]);
}

/* Eqs. (verletPos, verletVel) for one vertex with dt = 1: tentative
 * position from the interpolated fluid velocity U, velocity from the
 * three-level backward difference, then the position again with that
 * velocity.  Returns the new position and the velocity u(t+dt). */
void orc_verlet(const double *x, const double *xprev, const double *U, const double *acc, double *xnew,
                double *unew) {
    double xt[3];
    for (int k = 0; k < 3; ++k) xt[k] = x[k] + U[k] + 0.5 * acc[k];
    for (int k = 0; k < 3; ++k) unew[k] = 1.5 * xt[k] - 2.0 * x[k] + 0.5 * xprev[k];
    for (int k = 0; k < 3; ++k) xnew[k] = x[k] + unew[k] + 0.5 * acc[k];
}

/* ------------------------------------------------------------------------ */
/* Whole-method simulation state.                                            */
/* ------------------------------------------------------------------------ */
typedef struct {
    int rigid;
    double ks0, Eb, kv, thickness, density_ratio, ref_radius;
    double gravity[3], u0[3], omega0[3];
    int bend_variant;
    int kinematic; /* membrane: markers advected with the fluid (kinematic IB) */
    int rigid_force; /* rigid: 0 probe stress jump (as printed), 1 momentum exchange */
    int centroid_markers; /* 1: the IB markers are the triangle centroids (as printed in Sec. 2.3) */
    int mass_model; /* membrane mass: 0 a shell of thickness T and density rho_s (Sec. 3.5),
                       1 a capsule of density rho_s, i.e. rho_s times the enclosed volume (Sec. 3.4) */
} orc_body_params;

typedef struct {
    int rigid, nv, nt, nh;
    orc_body_params p;
    double *X, *Xprev;     /* [nv*3] */
    double *Xbody;         /* rigid: rest coordinates about the centroid */
    int *tri, *hinge;      /* [nt*3], [nh*4] */
    int *edge;             /* [nh*2] */
    double *ks, *l0, *kb, *theta0;
    double V0, A0, mv;
    double *Ub, *U, *Fl;   /* last step: boundary velocity, interpolated velocity, IB force */
    double *Uc, *Flc;      /* centroid markers [nt*3]: interpolated velocity, IB force */
    /* rigid state */
    double xc[3], q[4], u[3], up[3], w[3], wp[3], m, Vb, Ib[9];
} orc_body;

typedef struct {
    int n[3];
    long ncell;
    double tau, nu;
    double gext[3];
    int bc[3];
    double wall_u[6][3];
    double *fpost; /* post-collision populations, [ncell*19] */
    double *f;     /* streamed populations of the current step */
    double *rho, *us; /* predictor moments rho, u* of the current step */
    double *fib;      /* IB body force of the current step, [ncell*3] */
    double *rho_out, *u_out; /* moments of the last collision */
    orc_body *bodies;
    int nbody;
    long step;
    int err;
} orc_sim;

static long cell_index(const orc_sim *s, int x, int y, int z) {
    return (long)x + (long)s->n[0] * ((long)y + (long)s->n[1] * (long)z);
}

orc_sim *orc_sim_create(int nx, int ny, int nz, double tau, const double *gext, const int *bc,
                        const double *wall_u) {
    if (nx < 1 || ny < 1 || nz < 1 || !(tau > 0.5)) return NULL;
    for (int a = 0; a < 3; ++a)
        if (bc[a] == BC_WALL && (a == 0 ? nx : a == 1 ? ny : nz) < 3) return NULL;
    orc_sim *s = (orc_sim *)calloc(1, sizeof(orc_sim));
    s->n[0] = nx;
    s->n[1] = ny;
    s->n[2] = nz;
    s->ncell = (long)nx * ny * nz;
    s->tau = tau;
    s->nu = CS2 * (tau - 0.5); /* nu = c_s^2 (tau - dt/2), Sec. 2.1 */
    for (int a = 0; a < 3; ++a) {
        s->gext[a] = gext ? gext[a] : 0.0;
        s->bc[a] = bc[a];
    }
    for (int fc = 0; fc < 6; ++fc)
        for (int a = 0; a < 3; ++a) s->wall_u[fc][a] = wall_u ? wall_u[3 * fc + a] : 0.0;
    s->fpost = (double *)malloc(sizeof(double) * Q * s->ncell);
    s->f = (double *)malloc(sizeof(double) * Q * s->ncell);
    s->rho = (double *)malloc(sizeof(double) * s->ncell);
    s->us = (double *)malloc(sizeof(double) * 3 * s->ncell);
    s->fib = (double *)malloc(sizeof(double) * 3 * s->ncell);
    s->rho_out = (double *)malloc(sizeof(double) * s->ncell);
    s->u_out = (double *)malloc(sizeof(double) * 3 * s->ncell);
    if (!s->fpost || !s->f || !s->rho || !s->us || !s->fib || !s->rho_out || !s->u_out) return NULL;
    /* fluid at rest, rho = 1 */
    double u0[3] = {0, 0, 0}, feq[Q];
    orc_feq(1.0, u0, feq);
    for (long c = 0; c < s->ncell; ++c) {
        for (int i = 0; i < Q; ++i) s->fpost[c * Q + i] = feq[i];
        s->rho_out[c] = 1.0;
        for (int a = 0; a < 3; ++a) s->u_out[3 * c + a] = 0.0;
    }
    return s;
}

/* Initial condition: f = f^eq(rho(x), u(x)) (reading: the fluid starts at
 * equilibrium with the given fields). */
void orc_sim_set_fields(orc_sim *s, const double *rho, const double *u) {
    for (long c = 0; c < s->ncell; ++c) {
        orc_feq(rho[c], &u[3 * c], &s->fpost[c * Q]);
        s->rho_out[c] = rho[c];
        for (int a = 0; a < 3; ++a) s->u_out[3 * c + a] = u[3 * c + a];
    }
}

void orc_sim_set_populations(orc_sim *s, const double *f) {
    memcpy(s->fpost, f, sizeof(double) * Q * s->ncell);
}

void orc_sim_get_populations(const orc_sim *s, double *f) {
    memcpy(f, s->fpost, sizeof(double) * Q * s->ncell);
}

void orc_sim_get_fields(const orc_sim *s, double *rho, double *u) {
    if (rho) memcpy(rho, s->rho_out, sizeof(double) * s->ncell);
    if (u) memcpy(u, s->u_out, sizeof(double) * 3 * s->ncell);
}

static void body_free(orc_body *b) {
    free(b->X);
    free(b->Xprev);
    free(b->Xbody);
    free(b->tri);
    free(b->hinge);
    free(b->edge);
    free(b->ks);
    free(b->l0);
    free(b->kb);
    free(b->theta0);
    free(b->Ub);
    free(b->U);
    free(b->Fl);
    free(b->Uc);
    free(b->Flc);
}

void orc_sim_destroy(orc_sim *s) {
    if (!s) return;
    for (int b = 0; b < s->nbody; ++b) body_free(&s->bodies[b]);
    free(s->bodies);
    free(s->fpost);
    free(s->f);
    free(s->rho);
    free(s->us);
    free(s->fib);
    free(s->rho_out);
    free(s->u_out);
    free(s);
}

/* Adds a body given its vertices (markers, reading: markers are the mesh
 * vertices, where the network forces and the Newton equation act) and its
 * outward-oriented triangles.  Rest state, in FP64:
 *   spring constants k_{s,l} = k_{s,0} T (A_1 + A_2) / l0^2 (Van Gelder,
 *   Sec. 2.3; reading: rest areas and lengths), rest dihedral angles,
 *   k_b = Eb k_{s,l} r^2 per hinge (r = body radius), V0, rest area,
 *   vertex mass m_v = (rho_s/rho_f) T A_total / N_v (membrane mass spread
 *   uniformly, Sec. 2.3 and Sec. 3.5);
 *   rigid: volume, volume centroid, inertia tensor of the solid with density
 *   rho_s, rest coordinates about the centroid.
 * Returns the body index or a negative error. */
int orc_sim_add_body(orc_sim *s, const double *verts, int nv, const int *tris, int nt,
                     const orc_body_params *p) {
    if (nv < 4 || nt < 4) return ORC_EINVAL;
    orc_body b;
    memset(&b, 0, sizeof(b));
    b.p = *p;
    b.rigid = p->rigid;
    b.nv = nv;
    b.nt = nt;
    b.X = (double *)malloc(sizeof(double) * 3 * nv);
    b.Xprev = (double *)malloc(sizeof(double) * 3 * nv);
    b.tri = (int *)malloc(sizeof(int) * 3 * nt);
    memcpy(b.X, verts, sizeof(double) * 3 * nv);
    memcpy(b.Xprev, verts, sizeof(double) * 3 * nv); /* reading: x(t - dt) = x(t) at start */
    memcpy(b.tri, tris, sizeof(int) * 3 * nt);
    int *hinge = (int *)malloc(sizeof(int) * 4 * 3 * nt);
    int *htri = (int *)malloc(sizeof(int) * 2 * 3 * nt);
    int nh = orc_mesh_hinges(nv, nt, tris, hinge, htri);
    if (nh < 0) {
        free(hinge);
        free(htri);
        body_free(&b);
        return ORC_EINVAL;
    }
    b.nh = nh;
    b.hinge = hinge;
    b.edge = (int *)malloc(sizeof(int) * 2 * nh);
    b.ks = (double *)malloc(sizeof(double) * nh);
    b.l0 = (double *)malloc(sizeof(double) * nh);
    b.kb = (double *)malloc(sizeof(double) * nh);
    b.theta0 = (double *)malloc(sizeof(double) * nh);
    for (int h = 0; h < nh; ++h) {
        const int *v = &hinge[4 * h];
        b.edge[2 * h] = v[0];
        b.edge[2 * h + 1] = v[1];
        double r[3];
        sub3(&verts[3 * v[0]], &verts[3 * v[1]], r);
        double l = norm3(r);
        double n[3], A1, A2, c[3];
        tri_geom(verts, &tris[3 * htri[2 * h]], n, &A1, c);
        tri_geom(verts, &tris[3 * htri[2 * h + 1]], n, &A2, c);
        b.l0[h] = l;
        b.ks[h] = p->ks0 * p->thickness * (A1 + A2) / (l * l);
        b.kb[h] = p->Eb * b.ks[h] * p->ref_radius * p->ref_radius;
        b.theta0[h] = orc_hinge_theta(&verts[3 * v[0]], &verts[3 * v[1]], &verts[3 * v[2]], &verts[3 * v[3]], NULL);
    }
    free(htri);
    b.V0 = orc_volume(verts, nt, tris);
    b.A0 = orc_area(verts, nt, tris);
    if (!(b.V0 > 0.0)) {
        body_free(&b);
        return ORC_EINVAL;
    }
    /* membrane mass, uniform over the vertices (Eq. newtonSoft): the shell
     * of unit thickness of Sec. 3.5, or the capsule of unit density ratio of
     * Sec. 3.4, whose mass is that of its enclosed volume */
    b.mv = p->mass_model == 1 ? p->density_ratio * b.V0 / nv : p->density_ratio * p->thickness * b.A0 / nv;
    b.Ub = (double *)calloc(3 * (size_t)nv, sizeof(double));
    b.U = (double *)calloc(3 * (size_t)nv, sizeof(double));
    b.Fl = (double *)calloc(3 * (size_t)nv, sizeof(double));
    if (p->centroid_markers) {
        b.Uc = (double *)calloc(3 * (size_t)nt, sizeof(double));
        b.Flc = (double *)calloc(3 * (size_t)nt, sizeof(double));
    }
    if (b.rigid) {
        double V, c[3], I[9];
        orc_mass_properties(verts, nt, tris, &V, c, I);
        b.Vb = V;
        b.m = p->density_ratio * V;
        for (int k = 0; k < 9; ++k) b.Ib[k] = p->density_ratio * I[k];
        for (int k = 0; k < 3; ++k) {
            b.xc[k] = c[k];
            b.u[k] = b.up[k] = p->u0[k];     /* reading: u(t-dt) = u(t-2dt) = u0 */
            b.w[k] = b.wp[k] = p->omega0[k];
        }
        b.q[0] = 1.0;
        b.q[1] = b.q[2] = b.q[3] = 0.0;
        b.Xbody = (double *)malloc(sizeof(double) * 3 * nv);
        for (int v = 0; v < nv; ++v)
            for (int k = 0; k < 3; ++k) b.Xbody[3 * v + k] = verts[3 * v + k] - c[k];
    }
    s->bodies = (orc_body *)realloc(s->bodies, sizeof(orc_body) * (size_t)(s->nbody + 1));
    s->bodies[s->nbody] = b;
    return s->nbody++;
}

/* MLS at point X against a lattice of size n with boundary kinds bc: shape
 * functions plus the linear indices of the 27 support nodes (periodic axes
 * wrap).  reading: a support that reaches a wall node (index 0 or n-1 of a
 * walled axis) is an error. */
static int mls_support_on(const int *n, const int *bc, const double *X, double *psi, long *node) {
    int base[3];
    if (orc_mls_point(X, base, psi)) return ORC_EINVAL;
    for (int a = 0; a < 3; ++a)
        if (bc[a] == BC_WALL && (base[a] - 1 < 1 || base[a] + 1 > n[a] - 2)) return ORC_EBODY_WALL;
    for (int k = 0; k < 27; ++k) {
        int d[3] = {k % 3 - 1, (k / 3) % 3 - 1, k / 9 - 1}, c[3];
        for (int a = 0; a < 3; ++a) {
            c[a] = base[a] + d[a];
            if (bc[a] == BC_PERIODIC) c[a] = ((c[a] % n[a]) + n[a]) % n[a];
        }
        node[k] = (long)c[0] + (long)n[0] * ((long)c[1] + (long)n[1] * (long)c[2]);
    }
    return ORC_OK;
}

static int mls_support(const orc_sim *s, const double *X, double *psi, long *node) {
    return mls_support_on(s->n, s->bc, X, psi, node);
}

/* Hydrodynamic stresses on triangle t (Eqs. hydroForP, hydroForNu): probes
 * at the centroid +- 1.2 dx along the outward normal; at each probe the MLS
 * fit of rho and of the velocity gives p = c_s^2 rho and, reading, the
 * Newtonian stress tau = rho nu (grad u + grad u^T).
 * F = [-(p+ - p-) n + (tau+ - tau-) . n] A.
 * The nodal fields rho[ncell] and u[3*ncell] are those of the current step. */
int orc_hydro_force_fields(const int *n, const int *bc, double nu, const double *rho_f, const double *u_f,
                           const double *X, const int *t, double *F, double *cen_out) {
    double nrm[3], A, cen[3];
    tri_geom(X, t, nrm, &A, cen);
    double p_side[2], tn_side[2][3];
    for (int side = 0; side < 2; ++side) {
        double sgn = side == 0 ? 1.0 : -1.0, P[3];
        for (int a = 0; a < 3; ++a) P[a] = cen[a] + sgn * 1.2 * nrm[a];
        double psi[27 * 4];
        long node[27];
        int rc = mls_support_on(n, bc, P, psi, node);
        if (rc) return rc;
        double fr[4] = {0, 0, 0, 0}, fu[3][4] = {{0}};
        for (int k = 0; k < 27; ++k)
            for (int i = 0; i < 4; ++i) {
                fr[i] += psi[4 * k + i] * rho_f[node[k]];
                for (int j = 0; j < 3; ++j) fu[j][i] += psi[4 * k + i] * u_f[3 * node[k] + j];
            }
        double rho = fr[0];
        p_side[side] = CS2 * rho;
        for (int j = 0; j < 3; ++j) {
            double acc = 0.0;
            for (int m = 0; m < 3; ++m) {
                /* d u_j / d x_m = fu[j][m+1] */
                double tau_jm = rho * nu * (fu[j][m + 1] + fu[m][j + 1]);
                acc += tau_jm * nrm[m];
            }
            tn_side[side][j] = acc;
        }
    }
    for (int a = 0; a < 3; ++a)
        F[a] = (-(p_side[0] - p_side[1]) * nrm[a] + (tn_side[0][a] - tn_side[1][a])) * A;
    if (cen_out)
        for (int a = 0; a < 3; ++a) cen_out[a] = cen[a];
    return ORC_OK;
}

static int hydro_force(const orc_sim *s, const double *X, const int *t, double *F, double *cen_out) {
    return orc_hydro_force_fields(s->n, s->bc, s->nu, s->rho, s->us, X, t, F, cen_out);
}

/* One body's part of a step (Sec. 2.2 and 2.3), weak coupling: everything
 * uses the fluid state of level n; the IB force is added to s->fib. */
static int body_step(orc_sim *s, orc_body *b) {
    int nv = b->nv, nt = b->nt;
    /* the IB markers: the vertices, or (centroid_markers) the triangle
     * centroids, each carrying its share of the surface */
    const int cm = b->p.centroid_markers;
    const int nm = cm ? nt : nv;
    double *phi = (double *)malloc(sizeof(double) * 27 * nm);
    long *node = (long *)malloc(sizeof(long) * 27 * nm);
    double *Ftot = (double *)calloc(3 * (size_t)nv, sizeof(double));
    double *Xnew = (double *)malloc(sizeof(double) * 3 * nv);
    double *Av = (double *)calloc((size_t)nv, sizeof(double));
    double *At = (double *)malloc(sizeof(double) * nt);
    double *Ftri = (double *)malloc(sizeof(double) * 3 * nt);
    double *cen = (double *)malloc(sizeof(double) * 3 * nt);
    double *Ubc = cm ? (double *)malloc(sizeof(double) * 3 * nt) : NULL;
    int rc = ORC_OK;

    /* (1) MLS interpolation of the fluid velocity at each marker, Eq. (uLag). */
    for (int l = 0; l < nm && !rc; ++l) {
        double psi[27 * 4], Xl[3];
        for (int a = 0; a < 3; ++a)
            Xl[a] = cm ? (b->X[3 * b->tri[3 * l] + a] + b->X[3 * b->tri[3 * l + 1] + a] +
                          b->X[3 * b->tri[3 * l + 2] + a]) / 3.0
                       : b->X[3 * l + a];
        rc = mls_support(s, Xl, psi, &node[27 * l]);
        if (rc) break;
        double U[3] = {0, 0, 0};
        for (int k = 0; k < 27; ++k) {
            phi[27 * l + k] = psi[4 * k];
            for (int a = 0; a < 3; ++a) U[a] += psi[4 * k] * s->us[3 * node[27 * l + k] + a];
        }
        for (int a = 0; a < 3; ++a) (cm ? b->Uc : b->U)[3 * l + a] = U[a];
    }
    /* (2) geometry at level n: vertex areas 1/3 sum of incident areas, and
     * the hydrodynamic force of each element (Eqs. hydroForP, hydroForNu). */
    for (int t = 0; t < nt && !rc; ++t) {
        double n[3], A, c[3];
        tri_geom(b->X, &b->tri[3 * t], n, &A, c);
        At[t] = A;
        for (int q = 0; q < 3; ++q) Av[b->tri[3 * t + q]] += A / 3.0;
        rc = hydro_force(s, b->X, &b->tri[3 * t], &Ftri[3 * t], &cen[3 * t]);
    }
    if (rc) goto done;
    if (cm) {
        /* reading (centroid markers): a vertex moves with the mean of its
         * triangles' centroid velocities, each weighted by the third of the
         * triangle's area the vertex carries */
        for (int l = 0; l < 3 * nv; ++l) b->U[l] = 0.0;
        for (int t = 0; t < nt; ++t)
            for (int q = 0; q < 3; ++q)
                for (int a = 0; a < 3; ++a) b->U[3 * b->tri[3 * t + q] + a] += At[t] / 3.0 * b->Uc[3 * t + a];
        for (int l = 0; l < nv; ++l)
            for (int a = 0; a < 3; ++a) b->U[3 * l + a] /= Av[l];
    }

    double *Ub = b->Ub;
    if (!b->rigid) {
        /* (3) internal forces (Eqs. strainFor, bendFor, volFor) plus the
         * element hydrodynamic forces shared 1/3 per vertex (Eq. newtonSoft). */
        orc_spring_forces(b->X, b->nh, b->edge, b->ks, b->l0, Ftot);
        orc_bend_forces(b->X, b->nh, b->hinge, b->kb, b->theta0, b->p.bend_variant, Ftot);
        orc_volume_forces(b->X, nt, b->tri, b->p.kv, b->V0, Ftot);
        if (!b->p.kinematic)
            for (int t = 0; t < nt; ++t)
                for (int q = 0; q < 3; ++q)
                    for (int a = 0; a < 3; ++a) Ftot[3 * b->tri[3 * t + q] + a] += Ftri[3 * t + a] / 3.0;
        /* (4) Verlet with the interpolated velocity as tentative velocity
         * (Eqs. verletPos, verletVel) moves the vertices.  reading: the
         * boundary velocity imposed by the IB force is the tentative
         * velocity advanced by Newton's law over one step,
         * U_b = U + (F_tot/m_v) dt, so that F_l = F_tot/m_v.  Imposing the
         * backward-difference velocity instead makes even a force-free
         * membrane drive the fluid (F_l = (U - u(t-dt))/2), and that
         * feedback grows without bound on the lattice. */
        for (int l = 0; l < nv; ++l) {
            double acc[3], xn[3], ubdf[3];
            for (int a = 0; a < 3; ++a) acc[a] = Ftot[3 * l + a] / b->mv;
            if (b->p.kinematic) {
                /* kinematic IB (the variant of Sec. 3.4): the vertices are
                 * advected with the interpolated fluid velocity, X += U dt;
                 * the fluid feels the membrane's internal forces alone (the
                 * element hydrodynamic stresses are the fluid's own) */
                for (int a = 0; a < 3; ++a) xn[a] = b->X[3 * l + a] + b->U[3 * l + a];
            } else {
                orc_verlet(&b->X[3 * l], &b->Xprev[3 * l], &b->U[3 * l], acc, xn, ubdf);
            }
            for (int a = 0; a < 3; ++a) {
                Xnew[3 * l + a] = xn[a];
                Ub[3 * l + a] = b->U[3 * l + a] + acc[a];
            }
        }
    } else {
        /* (3') rigid body: total force and moment of the element stresses,
         * plus reading: gravity minus buoyancy (rho_s - rho_f) V g. */
        double F[3] = {0, 0, 0}, M[3] = {0, 0, 0};
        if (!b->p.rigid_force) {
            for (int t = 0; t < nt; ++t) {
                double r[3], rxF[3];
                sub3(&cen[3 * t], b->xc, r);
                cross3(r, &Ftri[3 * t], rxF);
                for (int a = 0; a < 3; ++a) {
                    F[a] += Ftri[3 * t + a];
                    M[a] += rxF[a];
                }
            }
        } else {
            /* reading (momentum exchange, the alternative to the printed
             * stress jump): the fluid pushes back with minus the IB force it
             * received in the previous step, -sum_l A_l F_l and its moment,
             * plus the rate of change of the momentum of the fluid inside the
             * body moving with it, rho_f V du/dt and I_f dw/dt (backward
             * differences, I_f the body's world-frame inertia scaled by
             * rho_f / rho_s) */
            for (int l = 0; l < nm; ++l) {
                double r[3], f[3], rxf[3];
                sub3(cm ? &cen[3 * l] : &b->X[3 * l], b->xc, r);
                for (int a = 0; a < 3; ++a) f[a] = cm ? -At[l] * b->Flc[3 * l + a] : -Av[l] * b->Fl[3 * l + a];
                cross3(r, f, rxf);
                for (int a = 0; a < 3; ++a) {
                    F[a] += f[a];
                    M[a] += rxf[a];
                }
            }
            double Rq[9], dw_body[3], Idw[3];
            quat_to_R(b->q, Rq);
            /* I_world (w - wp) = R I_b R^T (w - wp) */
            for (int i = 0; i < 3; ++i)
                dw_body[i] = Rq[i] * (b->w[0] - b->wp[0]) + Rq[3 + i] * (b->w[1] - b->wp[1]) +
                             Rq[6 + i] * (b->w[2] - b->wp[2]);
            for (int i = 0; i < 3; ++i)
                Idw[i] = b->Ib[3 * i] * dw_body[0] + b->Ib[3 * i + 1] * dw_body[1] + b->Ib[3 * i + 2] * dw_body[2];
            for (int a = 0; a < 3; ++a) {
                F[a] += b->Vb * (b->u[a] - b->up[a]);
                M[a] += (Rq[3 * a] * Idw[0] + Rq[3 * a + 1] * Idw[1] + Rq[3 * a + 2] * Idw[2]) / b->p.density_ratio;
            }
        }
        for (int a = 0; a < 3; ++a) F[a] += (b->p.density_ratio - 1.0) * b->Vb * b->p.gravity[a];
        /* F = m du/dt, M = I dw/dt with I in the world frame (reading: no
         * gyroscopic term, as printed). */
        double R[9], Iw[9], Iwi[9], tmp[9];
        quat_to_R(b->q, R);
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k) acc += R[3 * i + k] * b->Ib[3 * k + j];
                tmp[3 * i + j] = acc;
            }
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                double acc = 0.0;
                for (int k = 0; k < 3; ++k) acc += tmp[3 * i + k] * R[3 * j + k];
                Iw[3 * i + j] = acc;
            }
        inverse3(Iw, Iwi);
        double udot[3], wdot[3];
        for (int a = 0; a < 3; ++a) {
            udot[a] = F[a] / b->m;
            wdot[a] = Iwi[3 * a] * M[0] + Iwi[3 * a + 1] * M[1] + Iwi[3 * a + 2] * M[2];
        }
        double un[3], wn[3];
        orc_bdf2(b->u, b->up, udot, un);
        orc_bdf2(b->w, b->wp, wdot, wn);
        /* boundary velocity of each marker at level n: u + w x (X - x_c) */
        for (int l = 0; l < nv; ++l) {
            double r[3], wxr[3];
            sub3(&b->X[3 * l], b->xc, r);
            cross3(wn, r, wxr);
            for (int a = 0; a < 3; ++a) Ub[3 * l + a] = un[a] + wxr[a];
        }
        if (cm)
            for (int t = 0; t < nt; ++t) {
                double r[3], wxr[3];
                sub3(&cen[3 * t], b->xc, r);
                cross3(wn, r, wxr);
                for (int a = 0; a < 3; ++a) Ubc[3 * t + a] = un[a] + wxr[a];
            }
        /* advance centre and orientation (reading: x_c += u dt; exact
         * rotation by |w| dt about w), then the markers */
        for (int a = 0; a < 3; ++a) {
            b->xc[a] += un[a];
            b->up[a] = b->u[a];
            b->u[a] = un[a];
            b->wp[a] = b->w[a];
            b->w[a] = wn[a];
        }
        double wl = norm3(wn);
        if (wl > 0.0) {
            double dq[4] = {cos(0.5 * wl), sin(0.5 * wl) * wn[0] / wl, sin(0.5 * wl) * wn[1] / wl,
                            sin(0.5 * wl) * wn[2] / wl};
            double qn[4];
            quat_mul(dq, b->q, qn);
            double qq = sqrt(qn[0] * qn[0] + qn[1] * qn[1] + qn[2] * qn[2] + qn[3] * qn[3]);
            for (int k = 0; k < 4; ++k) b->q[k] = qn[k] / qq;
        }
        quat_to_R(b->q, R);
        for (int l = 0; l < nv; ++l) {
            for (int a = 0; a < 3; ++a)
                Xnew[3 * l + a] = b->xc[a] + R[3 * a] * b->Xbody[3 * l] + R[3 * a + 1] * b->Xbody[3 * l + 1] +
                                  R[3 * a + 2] * b->Xbody[3 * l + 2];
        }
    }
    /* (5) Lagrangian force F_l = (U_b - U)/dt and spreading, Eq. (bodyforce),
     * with the shape functions of level n.  reading: c_l = A_l, the marker's
     * share of the surface (volume A_l dx over a cell dx^3), which makes the
     * Eulerian total equal sum_l c_l F_l since sum_k phi_k = 1. */
    for (int l = 0; l < nv; ++l)
        for (int a = 0; a < 3; ++a) b->Fl[3 * l + a] = Ub[3 * l + a] - b->U[3 * l + a];
    if (cm && !b->rigid)
        /* centroid markers of a membrane: the boundary velocity at a
         * centroid is its interpolated velocity advanced by the mean
         * Newton acceleration of the triangle's vertices */
        for (int t = 0; t < nt; ++t)
            for (int a = 0; a < 3; ++a) {
                double acc = 0.0;
                for (int q = 0; q < 3; ++q) acc += b->Fl[3 * b->tri[3 * t + q] + a];
                Ubc[3 * t + a] = b->Uc[3 * t + a] + acc / 3.0;
            }
    for (int l = 0; l < nm; ++l) {
        double Fl[3];
        for (int a = 0; a < 3; ++a) {
            Fl[a] = cm ? Ubc[3 * l + a] - b->Uc[3 * l + a] : b->Fl[3 * l + a];
            if (cm) b->Flc[3 * l + a] = Fl[a];
        }
        const double cl = cm ? At[l] : Av[l];
        for (int k = 0; k < 27; ++k) {
            long c = node[27 * l + k];
            for (int a = 0; a < 3; ++a) s->fib[3 * c + a] += cl * phi[27 * l + k] * Fl[a];
        }
    }
    /* (6) shift the marker history: x(t - dt) <- x(t), x(t) <- x(t + dt) */
    for (int l = 0; l < 3 * nv; ++l) {
        b->Xprev[l] = b->X[l];
        b->X[l] = Xnew[l];
    }
done:
    free(Xnew);
    free(phi);
    free(node);
    free(Ftot);
    free(Av);
    free(At);
    free(Ftri);
    free(cen);
    free(Ubc);
    return rc;
}

/* Lists the walls a node lies on; face index fc = 2a + (s<0). */
static int node_walls(const orc_sim *s, const int *c, int *axes, int *signs) {
    int nf = 0;
    for (int a = 0; a < 3; ++a) {
        if (s->bc[a] != BC_WALL) continue;
        if (c[a] == 0) {
            axes[nf] = a;
            signs[nf++] = +1;
        } else if (c[a] == s->n[a] - 1) {
            axes[nf] = a;
            signs[nf++] = -1;
        }
    }
    return nf;
}

/* Streaming (left-hand side of Eq. evoleq, pull form f_i(x) = f*_i(x - e_i))
 * with periodic wrap, then the wall rules, then the predictor moments
 * rho = sum f and rho u* = sum f e + g_ext/2 (g_ext = 0 on wall nodes). */
static void stream_and_predict(orc_sim *s) {
    const int nx = s->n[0], ny = s->n[1], nz = s->n[2];
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int c[3] = {x, y, z};
                long idx = cell_index(s, x, y, z);
                double *f = &s->f[idx * Q];
                for (int i = 0; i < Q; ++i) {
                    int src[3], known = 1;
                    for (int a = 0; a < 3; ++a) {
                        src[a] = c[a] - E[i][a];
                        if (src[a] < 0 || src[a] >= s->n[a]) {
                            if (s->bc[a] == BC_PERIODIC)
                                src[a] = (src[a] + s->n[a]) % s->n[a];
                            else
                                known = 0;
                        }
                    }
                    f[i] = known ? s->fpost[cell_index(s, src[0], src[1], src[2]) * Q + i] : NAN;
                }
                int axes[3], signs[3];
                int nf = node_walls(s, c, axes, signs);
                if (nf == 1) {
                    orc_zouhe_face(f, axes[0], signs[0], s->wall_u[2 * axes[0] + (signs[0] < 0)]);
                } else if (nf > 1) {
                    double uwf[9];
                    for (int j = 0; j < nf; ++j)
                        for (int a = 0; a < 3; ++a) uwf[3 * j + a] = s->wall_u[2 * axes[j] + (signs[j] < 0)][a];
                    orc_wall_multi(f, nf, axes, signs, uwf);
                }
                double rho = 0.0, m[3] = {0, 0, 0};
                for (int i = 0; i < Q; ++i) {
                    rho += f[i];
                    for (int a = 0; a < 3; ++a) m[a] += f[i] * E[i][a];
                }
                s->rho[idx] = rho;
                for (int a = 0; a < 3; ++a)
                    s->us[3 * idx + a] = (m[a] + (nf ? 0.0 : 0.5 * s->gext[a])) / rho;
                for (int a = 0; a < 3; ++a) s->fib[3 * idx + a] = 0.0;
            }
}

/* Collision of Eq. (evoleq) with f_lb = g_ext + f_ib (zero on wall nodes,
 * reading: the walls carry no body force). */
static void collide_all(orc_sim *s) {
    const int nx = s->n[0], ny = s->n[1], nz = s->n[2];
#pragma omp parallel for schedule(static)
    for (int z = 0; z < nz; ++z)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                int c[3] = {x, y, z}, axes[3], signs[3];
                long idx = cell_index(s, x, y, z);
                int nf = node_walls(s, c, axes, signs);
                double flb[3];
                for (int a = 0; a < 3; ++a) flb[a] = nf ? 0.0 : s->gext[a] + s->fib[3 * idx + a];
                double *f = &s->f[idx * Q];
                orc_collide(f, s->tau, flb, &s->rho_out[idx], &s->u_out[3 * idx]);
                for (int i = 0; i < Q; ++i) s->fpost[idx * Q + i] = f[i];
            }
}

/* Streaming and predictor moments only (used by tests of the probe force). */
void orc_sim_predict(orc_sim *s) { stream_and_predict(s); }

/* n time steps.  Order (Sec. 2.2, weak coupling of Sec. 2.3): stream and
 * wall rules, predictor moments, for each body the MLS interpolation,
 * structure forces, update and spreading, then the forced collision.
 * reading: the interpolated velocity is the IB-free predictor u*, and the
 * collision uses u = u* + f_ib/(2 rho), i.e. (sum f e + f_lb/2)/rho.
 * Returns 0 or the first error; errors are sticky. */
int orc_sim_step(orc_sim *s, int nsteps) {
    if (s->err) return s->err;
    for (int it = 0; it < nsteps; ++it) {
        stream_and_predict(s);
        for (int b = 0; b < s->nbody; ++b) {
            int rc = body_step(s, &s->bodies[b]);
            if (rc) {
                s->err = rc;
                return rc;
            }
        }
        collide_all(s);
        s->step++;
    }
    return ORC_OK;
}

int orc_sim_get_markers(const orc_sim *s, int body, double *X, double *V, double *F) {
    if (body < 0 || body >= s->nbody) return ORC_EINVAL;
    const orc_body *b = &s->bodies[body];
    if (X) memcpy(X, b->X, sizeof(double) * 3 * b->nv);
    if (V) memcpy(V, b->Ub, sizeof(double) * 3 * b->nv);
    if (F) memcpy(F, b->Fl, sizeof(double) * 3 * b->nv);
    return ORC_OK;
}

/* Body summary: xc[3], u[3], omega[3], q[4], volume, area.  Membranes report
 * the vertex mean and mean boundary velocity as xc and u. */
int orc_sim_get_body(const orc_sim *s, int body, double *out) {
    if (body < 0 || body >= s->nbody) return ORC_EINVAL;
    const orc_body *b = &s->bodies[body];
    memset(out, 0, sizeof(double) * 15);
    if (b->rigid) {
        for (int a = 0; a < 3; ++a) {
            out[a] = b->xc[a];
            out[3 + a] = b->u[a];
            out[6 + a] = b->w[a];
        }
        for (int k = 0; k < 4; ++k) out[9 + k] = b->q[k];
    } else {
        for (int l = 0; l < b->nv; ++l)
            for (int a = 0; a < 3; ++a) {
                out[a] += b->X[3 * l + a] / b->nv;
                out[3 + a] += b->Ub[3 * l + a] / b->nv;
            }
        out[9] = 1.0;
    }
    out[13] = orc_volume(b->X, b->nt, b->tri);
    out[14] = orc_area(b->X, b->nt, b->tri);
    return ORC_OK;
}

/* Rest-state arrays of a body, for tests: ks, l0, kb, theta0 per hinge,
 * the hinge list, and scalars (V0, A0, mv, m, Vb). */
int orc_sim_body_rest(const orc_sim *s, int body, int *hinge, double *ks, double *l0, double *kb,
                      double *theta0, double *scalars) {
    if (body < 0 || body >= s->nbody) return ORC_EINVAL;
    const orc_body *b = &s->bodies[body];
    if (hinge) memcpy(hinge, b->hinge, sizeof(int) * 4 * b->nh);
    if (ks) memcpy(ks, b->ks, sizeof(double) * b->nh);
    if (l0) memcpy(l0, b->l0, sizeof(double) * b->nh);
    if (kb) memcpy(kb, b->kb, sizeof(double) * b->nh);
    if (theta0) memcpy(theta0, b->theta0, sizeof(double) * b->nh);
    if (scalars) {
        scalars[0] = b->V0;
        scalars[1] = b->A0;
        scalars[2] = b->mv;
        scalars[3] = b->m;
        scalars[4] = b->Vb;
    }
    return b->nh;
}

long orc_sim_step_count(const orc_sim *s) { return s->step; }

/* predictor fields of the last step, for tests */
void orc_sim_get_predictor(const orc_sim *s, double *rho, double *us) {
    if (rho) memcpy(rho, s->rho, sizeof(double) * s->ncell);
    if (us) memcpy(us, s->us, sizeof(double) * 3 * s->ncell);
}

/* IB force field of the last step, for tests */
void orc_sim_get_fib(const orc_sim *s, double *fib) { memcpy(fib, s->fib, sizeof(double) * 3 * s->ncell); }
