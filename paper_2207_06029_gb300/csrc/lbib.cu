// liblbib C ABI (include/lbib.h): context, device memory, body set-up and
// the per-step launch sequence.  Host-side rest-state computations (mesh
// hinges, spring and bending constants, mass properties) are FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <array>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/lbib.h"
#include "lbib_device.cuh"
#include "lbib_kernels.h"

using namespace lbib;

namespace {

std::string g_create_error;

struct DevBody {
    int nv = 0, nt = 0, nh = 0, rigid = 0;
    lbib_body_params p{};
    double *X[3] = {nullptr, nullptr, nullptr};  // rotating buffers: prev, cur, next
    int cur = 1;
    double *U = nullptr, *Ub = nullptr, *Fl = nullptr, *tri_vol = nullptr;
    double *Uc = nullptr, *Flc = nullptr;  // centroid markers
    void *phi = nullptr, *tri_geo = nullptr, *probe = nullptr;  // arithmetic precision R
    void *Xrel[2] = {nullptr, nullptr};                          // R: X - origin, current and next
    float *Xlo[2] = {nullptr, nullptr};  // FP32 membranes: (X - origin) - Xrel, current and next
    int *perm = nullptr;  // MLS points (markers, probes) in cell order
    int *node = nullptr, *tri = nullptr, *vh_ptr = nullptr, *vh_list = nullptr, *vt_ptr = nullptr,
        *vt_list = nullptr;
    int4 *hinge = nullptr;
    void *ks = nullptr, *l0 = nullptr, *kb = nullptr, *theta0 = nullptr;  // R per hinge
    double *Xbody = nullptr, *rstate = nullptr;
    int *bbox[2] = {nullptr, nullptr};  // support-region node boxes, current and next
    int bcur = 0;
    double *vol_part = nullptr, *vol_sum = nullptr;
    unsigned int *vol_count = nullptr;
    int4 *vh_verts = nullptr;
    void *vh_par = nullptr;
    int nvol_part = 0;
    double V0 = 0, A0 = 0, mv = 0, origin[3] = {0, 0, 0};
};

struct Ctx {
    lbib_params p{};
    Lattice L{};
    int prec = 1;
    size_t elem = 4, relem = 4;
    void *fA = nullptr, *fB = nullptr, *force = nullptr, *fields = nullptr, *mom = nullptr;
    int nsm = 1;
    int fields_every = 0;  // <0 never, 0 last step of each lbib_step call, k>0 every k-th step
    uint32_t *stamp = nullptr;
    int ntiles = 0;
    int *d_err = nullptr;
    int *h_err = nullptr;
    double *scratch = nullptr;
    size_t scratch_bytes = 0;
    cudaStream_t stream = nullptr;           // the caller's (or the library's) stream
    cudaStream_t s_hi = nullptr, s_lo = nullptr;  // step streams: IB + box sweep (high priority), far field (low)
    cudaEvent_t ev_fork = nullptr, ev_far = nullptr, ev_near = nullptr, ev_join = nullptr;
    bool split_sweep = true;
    int ib_per_sm = 0;  // > 0: the IB kernels keep at most this many blocks per SM (lbib_set_ib_blocks)
    bool own_stream = false;
    std::vector<DevBody> bodies;
    uint32_t *d_step = nullptr;  // device step counter (tile flags of the IB force)
    uint32_t step_host = 0;      // host mirror of *d_step
    uint32_t *d_sr = nullptr;    // two-word seed counter of the stochastic rounding (bfloat16 storage)
    double *d_tot = nullptr;     // partials, counter and result of the FP64 mass/momentum totals
    double *d_watch = nullptr;   // divergence watchdog: mass of its first check, mass of its last
    int watch_every = 1000;      // watchdog cadence in steps (0: off)
    double watch_tol = 0.1;      // relative total-mass drift the watchdog tolerates
    // CUDA graphs of one step, one per phase of the buffer rotation (period 6)
    cudaStream_t s_cap = nullptr;
    cudaGraphExec_t gexec[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    bool graphs_valid = false, use_graphs = true, graphs_timed = false;
    long long graph_origin = 0;
    cudaEvent_t gev[6][6] = {};  // timing events recorded by the graphs
    bool gev_pending[6] = {false, false, false, false, false, false};
    double prof_acc[4] = {0.0, 0.0, 0.0, 0.0};
    long long prof_n = 0;
    long long steps = 0, launches = 0;
    int err = 0;
    std::string msg;
    size_t bytes = 0;
    std::vector<std::pair<void *, size_t>> allocs;
    double *mstage = nullptr;  // lbib_step_markers: device staging of the recorded markers
    size_t mstage_bytes = 0;
    std::vector<void *> transient;  // allocations a checkpoint leaves out (scratch, support moments)
    bool profile = false;
    std::vector<cudaEvent_t> events;  // per step: begin, after MLS, after structure, after sweep
    size_t nev = 0;
};

int fail(Ctx *c, int code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    c->msg = buf;
    return code;
}

int cuda_fail(Ctx *c, cudaError_t e, const char *what) {
    c->err = LBIB_ECUDA;
    return fail(c, LBIB_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

void *dev_alloc(Ctx *c, size_t bytes) {
    if (bytes == 0) bytes = 16;
    void *ptr = nullptr;
    if (c->p.alloc) {
        ptr = c->p.alloc(bytes, c->p.alloc_user);
        if (ptr && (reinterpret_cast<uintptr_t>(ptr) & 255)) {
            if (c->p.free) c->p.free(ptr, c->p.alloc_user);
            ptr = nullptr;
        }
    } else if (cudaMalloc(&ptr, bytes) != cudaSuccess) {
        cudaGetLastError();
        ptr = nullptr;
    }
    if (ptr) {
        c->allocs.push_back({ptr, bytes});
        c->bytes += bytes;
    }
    return ptr;
}

// Frees one block of dev_alloc (the caller has synchronised its uses).
void dev_free_one(Ctx *c, void *ptr) {
    for (size_t k = 0; k < c->allocs.size(); ++k)
        if (c->allocs[k].first == ptr) {
            if (c->p.free)
                c->p.free(ptr, c->p.alloc_user);
            else
                cudaFree(ptr);
            c->bytes -= c->allocs[k].second;
            c->allocs.erase(c->allocs.begin() + k);
            return;
        }
}

void dev_free_all(Ctx *c) {
    for (auto &a : c->allocs) {
        if (c->p.free)
            c->p.free(a.first, c->p.alloc_user);
        else
            cudaFree(a.first);
    }
    c->allocs.clear();
    c->bytes = 0;
}

template <typename T>
T *upload(Ctx *c, const std::vector<T> &v, int *rc) {
    T *d = (T *)dev_alloc(c, v.size() * sizeof(T));
    if (!d) {
        *rc = LBIB_ENOMEM;
        return nullptr;
    }
    if (!v.empty()) {
        cudaError_t e = cudaMemcpyAsync(d, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) {
            *rc = LBIB_ECUDA;
            return nullptr;
        }
    }
    return d;
}

// Uploads doubles in the arithmetic precision of the context.
void *upload_r(Ctx *c, const std::vector<double> &v, int *rc) {
    if (c->relem == 8) return upload(c, v, rc);
    std::vector<float> f(v.begin(), v.end());
    return upload(c, f, rc);
}

// Largest squared distance d2 for which sqrt(d2)/r_w <= 1 holds in IEEE
// double arithmetic, i.e. the MLS support cut-off of Eq. (intKernel)
// expressed on the squared distance (bisection on the bit patterns).
double mls_dist2_cut() {
    double lo = 1.0, hi = 4.0;
    uint64_t a, b;
    std::memcpy(&a, &lo, 8);
    std::memcpy(&b, &hi, 8);
    while (b - a > 1) {
        uint64_t m = a + (b - a) / 2;
        double d;
        std::memcpy(&d, &m, 8);
        if (std::sqrt(d) / 1.3 <= 1.0)
            a = m;
        else
            b = m;
    }
    double out;
    std::memcpy(&out, &a, 8);
    return out;
}

Ctx *as_ctx(void *h) { return static_cast<Ctx *>(h); }

void invalidate_graphs(Ctx *c);

// ---- host geometry (FP64) ----
inline void v_sub(const double *a, const double *b, double *o) {
    for (int i = 0; i < 3; ++i) o[i] = a[i] - b[i];
}
inline void v_cross(const double *a, const double *b, double *o) {
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}
inline double v_dot(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }

double tri_area(const double *X, const int *t) {
    double e1[3], e2[3], N[3];
    v_sub(X + 3 * t[1], X + 3 * t[0], e1);
    v_sub(X + 3 * t[2], X + 3 * t[0], e2);
    v_cross(e1, e2, N);
    return 0.5 * std::sqrt(v_dot(N, N));
}

// signed dihedral angle between the outward normals of T1 = (a,b,c) and
// T2 = (b,a,d), positive on convex hinges
double dihedral(const double *xa, const double *xb, const double *xc, const double *xd) {
    double e[3], ac[3], ad[3], N1[3], N2[3], c12[3];
    v_sub(xb, xa, e);
    v_sub(xc, xa, ac);
    v_sub(xd, xa, ad);
    v_cross(e, ac, N1);
    v_cross(ad, e, N2);
    const double l1 = std::sqrt(v_dot(N1, N1)), l2 = std::sqrt(v_dot(N2, N2)), le = std::sqrt(v_dot(e, e));
    double n1[3], n2[3];
    for (int k = 0; k < 3; ++k) {
        n1[k] = N1[k] / l1;
        n2[k] = N2[k] / l2;
    }
    v_cross(n1, n2, c12);
    return std::atan2(v_dot(c12, e) / le, v_dot(n1, n2));
}

// volume, volume centroid and inertia (about the centroid, unit density) of
// the solid bounded by a closed outward triangulation, by tetrahedra from
// the origin
void mass_props(const double *X, int nt, const int *tri, double *V, double *cen, double *I) {
    double vol = 0, c[3] = {0, 0, 0}, C[9] = {0};
    for (int t = 0; t < nt; ++t) {
        const double *a = X + 3 * tri[3 * t], *b = X + 3 * tri[3 * t + 1], *d = X + 3 * tri[3 * t + 2];
        double bd[3];
        v_cross(b, d, bd);
        const double v = v_dot(a, bd) / 6.0;
        vol += v;
        double s[3];
        for (int k = 0; k < 3; ++k) {
            s[k] = a[k] + b[k] + d[k];
            c[k] += v * s[k] / 4.0;
        }
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                C[3 * i + j] += v / 20.0 * (a[i] * a[j] + b[i] * b[j] + d[i] * d[j] + s[i] * s[j]);
    }
    for (int k = 0; k < 3; ++k) c[k] /= vol;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) C[3 * i + j] -= vol * c[i] * c[j];
    const double tr = C[0] + C[4] + C[8];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) I[3 * i + j] = (i == j ? tr : 0.0) - C[3 * i + j];
    *V = vol;
    for (int k = 0; k < 3; ++k) cen[k] = c[k];
}

BodyView make_view(Ctx *c, DevBody &b) {
    BodyView v{};
    v.nv = b.nv;
    v.nt = b.nt;
    v.rigid = b.rigid;
    const int prev = (b.cur + 2) % 3, next = (b.cur + 1) % 3;
    v.X = b.X[b.cur];
    v.Xprev = b.X[prev];
    v.Xnew = b.X[next];
    v.U = b.U;
    v.Ub = b.Ub;
    v.Fl = b.Fl;
    v.centroid = b.p.centroid_markers;
    v.nm = b.p.centroid_markers ? b.nt : b.nv;
    v.Uc = b.Uc;
    v.Flc = b.Flc;
    v.phi = b.phi;
    v.node = b.node;
    v.perm = b.perm;
    v.tri = b.tri;
    v.tri_geo = b.tri_geo;
    v.tri_vol = b.tri_vol;
    v.probe = b.probe;
    v.Xrel = b.Xrel[b.bcur];
    v.Xrel_next = b.Xrel[1 - b.bcur];
    v.Xlo = b.Xlo[b.bcur];
    v.Xlo_next = b.Xlo[1 - b.bcur];
    v.vh_ptr = b.vh_ptr;
    v.vh_list = b.vh_list;
    v.vt_ptr = b.vt_ptr;
    v.vt_list = b.vt_list;
    v.hinge = b.hinge;
    v.ks = b.ks;
    v.l0 = b.l0;
    v.kb = b.kb;
    v.theta0 = b.theta0;
    v.V0 = b.V0;
    v.mv = b.mv;
    v.inv_mv = 1.0 / b.mv;
    v.inv_6V0 = 1.0 / (6.0 * b.V0);
    v.kv = b.p.kv;
    for (int a = 0; a < 3; ++a) v.origin[a] = b.origin[a];
    v.bend_variant = b.p.bend_variant;
    v.kinematic = b.p.kinematic;
    v.rigid_force = b.p.rigid_force;
    v.Xbody = b.Xbody;
    v.rstate = b.rstate;
    v.bbox = b.bbox[b.bcur];
    v.bbox_next = b.bbox[1 - b.bcur];
    v.vol_part = b.vol_part;
    v.nvol_part = b.nvol_part;
    v.vol_count = b.vol_count;
    v.vol_sum = b.vol_sum;
    v.vh_verts = b.vh_verts;
    v.vh_par = b.vh_par;
    v.err = c->d_err;
    return v;
}

int check_device_error(Ctx *c) {
    if (*c->h_err != 0 && c->err == 0) {
        c->err = *c->h_err;
        if (c->err == LBIB_EBODY_WALL)
            fail(c, c->err, "an MLS support (marker or probe) reached a wall node");
        else if (c->err == LBIB_ETIMEOUT)
            fail(c, c->err, "a bounded wait of the persistent batched step expired (the launch ended early)");
        else if (c->err == LBIB_EDIVERGED)
            fail(c, c->err,
                 "the run diverged: a non-finite, non-positive or supersonic node, a mass drift beyond the "
                 "watchdog tolerance, or a marker moving a lattice unit in one step");
        else
            fail(c, c->err, "device error %d (singular MLS moment matrix)", c->err);
    }
    return c->err;
}

// The device error word is read here, not after every step: a copy per
// lbib_step call would add a dependent transfer to each step.
int sync_ctx(Ctx *c) {
    cudaError_t e = cudaMemcpyAsync(c->h_err, c->d_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamSynchronize");
    return check_device_error(c);
}

// Errors after which the state can still be read (the run stopped, the
// device is fine).
bool readable_error(int rc) { return rc == LBIB_EBODY_WALL || rc == LBIB_EDIVERGED; }

// Queues the divergence watchdog on the populations of the last step
// (c->fA), on stream st.  Shares the totals scratch (same stream order).
int enqueue_watch(Ctx *c, cudaStream_t st) {
    const int n = totals_scratch_doubles();
    unsigned int *count = reinterpret_cast<unsigned int *>(c->d_tot + (n - 4));
    cudaError_t e = launch_watch(c->prec, c->fA, c->L, c->d_tot, count, c->d_watch, c->watch_tol, c->d_err, st);
    c->launches++;
    if (e != cudaSuccess) return cuda_fail(c, e, "watchdog kernel");
    return LBIB_OK;
}

double *get_scratch(Ctx *c, size_t bytes) {
    if (c->scratch_bytes >= bytes) return c->scratch;
    c->scratch = (double *)dev_alloc(c, bytes);
    if (c->scratch) c->transient.push_back(c->scratch);
    c->scratch_bytes = c->scratch ? bytes : 0;
    return c->scratch;
}

}  // namespace

extern "C" {

const char *lbib_last_error(const void *h) {
    if (!h) return g_create_error.c_str();
    return static_cast<const Ctx *>(h)->msg.c_str();
}

int lbib_create(const lbib_params *p, void **out) {
    if (!p || !out) {
        g_create_error = "null argument";
        return LBIB_EINVAL;
    }
    *out = nullptr;
    const int n[3] = {p->nx, p->ny, p->nz};
    for (int a = 0; a < 3; ++a) {
        if (n[a] < 1 || (p->bc[a] != LBIB_PERIODIC && p->bc[a] != LBIB_WALL)) {
            g_create_error = "lattice size must be >= 1 and bc PERIODIC or WALL";
            return LBIB_EINVAL;
        }
        if (p->bc[a] == LBIB_WALL && n[a] < 3) {
            g_create_error = "a walled axis needs at least 3 nodes";
            return LBIB_EINVAL;
        }
    }
    if (n[1] > 65535 || n[2] > 65535) {
        g_create_error = "ny and nz must be at most 65535";
        return LBIB_EINVAL;
    }
    if (!(p->tau > 0.5) || !std::isfinite(p->tau)) {
        g_create_error = "tau must be > 0.5";
        return LBIB_EINVAL;
    }
    if (p->precision < LBIB_FP64 || p->precision > LBIB_BF16_DEV) {
        g_create_error = "unknown precision";
        return LBIB_EINVAL;
    }
    if ((p->alloc == nullptr) != (p->free == nullptr)) {
        g_create_error = "alloc and free must be given together";
        return LBIB_EINVAL;
    }
    const long long ncell = (long long)n[0] * n[1] * n[2];
    if (ncell > (1LL << 30)) {
        g_create_error = "lattice too large (more than 2^30 nodes)";
        return LBIB_EINVAL;
    }
    Ctx *c = new Ctx();
    c->p = *p;
    c->prec = p->precision;
    c->elem = c->prec == LBIB_FP64 ? 8 : c->prec == LBIB_FP32 ? 4 : 2;
    c->relem = c->prec == LBIB_FP64 ? 8 : 4;
    Lattice &L = c->L;
    L.nx = n[0];
    L.ny = n[1];
    L.nz = n[2];
    L.ntx = (n[0] + kTile - 1) / kTile;
    L.nty = (n[1] + kTile - 1) / kTile;
    L.ntz = (n[2] + kTile - 1) / kTile;
    L.ncell = (int)ncell;
    L.stride = (ncell + 63) / 64 * 64;
    L.off32 = (long long)Q * L.stride <= 0xFFFFFFFFLL;
    L.sweep_vec = 0;  // the one-node sweep; the autotuner may pick the row-tile kernel
    for (int a = 0; a < 3; ++a) {
        L.bc[a] = p->bc[a];
        L.gext[a] = p->body_force[a];
    }
    L.tau = p->tau;
    for (int f = 0; f < 6; ++f)
        for (int a = 0; a < 3; ++a) L.wall_u[f][a] = p->wall_u[f][a];
    L.dist2_cut = mls_dist2_cut();
    L.dist2_cut_f = (float)L.dist2_cut;
    L.omega_d = 1.0 / p->tau;
    L.cF_d = 1.0 - 0.5 / p->tau;
    L.nu_d = (p->tau - 0.5) / 3.0;
    L.omega_f = (float)L.omega_d;
    L.cF_f = (float)L.cF_d;
    // c_dg = omega/12 rounded, c_ax = (omega - 8 c_dg)/2: 8 c_dg lies within
    // a factor two of omega, so the difference and the halving are exact
    L.codd_d[1] = L.omega_d / 12.0;
    L.codd_d[0] = (L.omega_d - 8.0 * L.codd_d[1]) * 0.5;
    L.codd_f[1] = L.omega_f / 12.0f;
    L.codd_f[0] = (L.omega_f - 8.0f * L.codd_f[1]) * 0.5f;
    L.nu_f = (float)L.nu_d;
    for (int a = 0; a < 3; ++a) {
        L.gext_d[a] = p->body_force[a];
        L.gext_f[a] = (float)p->body_force[a];
    }
    // wall velocity per combination of faces: the face's own velocity on a
    // face node; on edges and corners no flow through any of the node's
    // faces (a component along a face normal is that face's own), the mean
    // of the faces' velocities in the remaining directions
    for (int cz = 0; cz < 3; ++cz)
        for (int cy = 0; cy < 3; ++cy)
            for (int cx = 0; cx < 3; ++cx) {
                const int code[3] = {cx, cy, cz};
                int faces[3], nf = 0;
                for (int a = 0; a < 3; ++a)
                    if (code[a]) faces[nf++] = 2 * a + (code[a] == 2);
                double uw[3] = {0.0, 0.0, 0.0};
                for (int a = 0; a < 3; ++a) {
                    if (code[a]) {
                        uw[a] = p->wall_u[2 * a + (code[a] == 2)][a];
                        continue;
                    }
                    for (int j = 0; j < nf; ++j) uw[a] += p->wall_u[faces[j]][a] / nf;
                }
                const int wc = wall_code(cx, cy, cz);
                for (int a = 0; a < 3; ++a) {
                    L.uw_d[wc][a] = uw[a];
                    L.uw_f[wc][a] = (float)uw[a];
                }
            }
    c->ntiles = L.ntx * L.nty * L.ntz;

    cudaError_t e;
    if (p->stream) {
        c->stream = (cudaStream_t)p->stream;
    } else {
        e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            g_create_error = std::string("cudaStreamCreate: ") + cudaGetErrorString(e);
            delete c;
            return LBIB_ECUDA;
        }
        c->own_stream = true;
    }
    int prio_lo = 0, prio_hi = 0;
    cudaDeviceGetStreamPriorityRange(&prio_lo, &prio_hi);
    if (cudaStreamCreateWithPriority(&c->s_hi, cudaStreamNonBlocking, prio_hi) != cudaSuccess ||
        cudaStreamCreateWithPriority(&c->s_lo, cudaStreamNonBlocking, prio_lo) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_far, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_near, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c->ev_join, cudaEventDisableTiming) != cudaSuccess) {
        g_create_error = std::string("stream/event creation: ") + cudaGetErrorString(cudaGetLastError());
        lbib_destroy(c);
        return LBIB_ECUDA;
    }
    const size_t pop_bytes = (size_t)Q * L.stride * c->elem;
    c->fA = dev_alloc(c, pop_bytes);
    c->fB = dev_alloc(c, pop_bytes);
    c->force = dev_alloc(c, 3 * (size_t)L.stride * c->relem);
    c->fields = dev_alloc(c, 4 * (size_t)L.stride * c->relem);
    c->mom = dev_alloc(c, 4 * (size_t)L.stride * c->relem);
    c->transient.push_back(c->mom);
    {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&c->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || c->nsm < 1) {
            cudaGetLastError();
            c->nsm = 1;
        }
    }
    c->stamp = (uint32_t *)dev_alloc(c, sizeof(uint32_t) * (size_t)c->ntiles);
    c->d_err = (int *)dev_alloc(c, sizeof(int));
    c->d_step = (uint32_t *)dev_alloc(c, sizeof(uint32_t));
    c->d_sr = (uint32_t *)dev_alloc(c, 2 * sizeof(uint32_t));
    c->d_tot = (double *)dev_alloc(c, sizeof(double) * (size_t)totals_scratch_doubles());
    c->d_watch = (double *)dev_alloc(c, 2 * sizeof(double));
    if (!c->fA || !c->fB || !c->force || !c->fields || !c->mom || !c->stamp || !c->d_err || !c->d_step || !c->d_sr ||
        !c->d_tot || !c->d_watch) {
        g_create_error = "device allocation failed";
        lbib_destroy(c);
        return LBIB_ENOMEM;
    }
    if (cudaMallocHost(&c->h_err, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        g_create_error = "pinned host allocation failed";
        c->h_err = nullptr;
        lbib_destroy(c);
        return LBIB_ENOMEM;
    }
    *c->h_err = 0;
    e = cudaMemsetAsync(c->force, 0, 3 * (size_t)L.stride * c->relem, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->stamp, 0, sizeof(uint32_t) * (size_t)c->ntiles, c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_err, 0, sizeof(int), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_step, 0, sizeof(uint32_t), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_sr, 0, 2 * sizeof(uint32_t), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_tot, 0, sizeof(double) * (size_t)totals_scratch_doubles(), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_watch, 0, 2 * sizeof(double), c->stream);
    if (e == cudaSuccess) e = prepare_kernels();
    if (e == cudaSuccess) e = prepare_sweep_kernels();
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->s_cap, cudaStreamNonBlocking);
    for (int k = 0; k < 6 && e == cudaSuccess; ++k)
        for (int j = 0; j < 6 && e == cudaSuccess; ++j) e = cudaEventCreate(&c->gev[k][j]);
    if (e != cudaSuccess) {
        g_create_error = std::string("cudaMemset: ") + cudaGetErrorString(e);
        lbib_destroy(c);
        return LBIB_ECUDA;
    }
    // fluid at rest, formed on the device (deviations f - w of zero)
    e = launch_init_equilibrium(c->prec, c->fA, c->L, nullptr, nullptr, c->fields, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) {
        g_create_error = std::string("initial state: ") + cudaGetErrorString(e);
        lbib_destroy(c);
        return LBIB_ECUDA;
    }
    c->launches++;
    *out = c;
    return LBIB_OK;
}

void lbib_destroy(void *h) {
    if (!h) return;
    Ctx *c = as_ctx(h);
    if (c->stream) cudaStreamSynchronize(c->stream);
    for (cudaStream_t st : {c->s_hi, c->s_lo})
        if (st) cudaStreamSynchronize(st);
    for (auto ev : c->events) cudaEventDestroy(ev);
    for (int k = 0; k < 6; ++k) {
        if (c->gexec[k]) cudaGraphExecDestroy(c->gexec[k]);
        for (int j = 0; j < 6; ++j)
            if (c->gev[k][j]) cudaEventDestroy(c->gev[k][j]);
    }
    if (c->s_cap) cudaStreamDestroy(c->s_cap);
    for (cudaEvent_t ev : {c->ev_fork, c->ev_far, c->ev_near, c->ev_join})
        if (ev) cudaEventDestroy(ev);
    for (cudaStream_t st : {c->s_hi, c->s_lo})
        if (st) cudaStreamDestroy(st);
    dev_free_all(c);
    if (c->h_err) cudaFreeHost(c->h_err);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

int lbib_set_shear_fields(void *h, double u_lo, double u_hi) {
    Ctx *c = as_ctx(h);
    if (!c) return LBIB_EINVAL;
    if (!std::isfinite(u_lo) || !std::isfinite(u_hi)) return fail(c, LBIB_EINVAL, "shear velocities must be finite");
    cudaError_t e = launch_init_equilibrium(c->prec, c->fA, c->L, nullptr, nullptr, c->fields, c->stream, u_lo, u_hi);
    c->launches++;
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_watch, 0, 2 * sizeof(double), c->stream);  // new reference mass
    if (e != cudaSuccess) return cuda_fail(c, e, "init kernel");
    return LBIB_OK;
}

int lbib_set_fields(void *h, const double *rho, const double *u, int on_device) {
    Ctx *c = as_ctx(h);
    if (!c || !rho || !u) return LBIB_EINVAL;
    const size_t n = (size_t)c->L.ncell;
    const double *drho = rho, *du = u;
    if (!on_device) {
        double *tmp = get_scratch(c, 4 * n * sizeof(double));
        if (!tmp) return fail(c, LBIB_ENOMEM, "scratch allocation failed");
        cudaError_t e = cudaMemcpyAsync(tmp, rho, n * sizeof(double), cudaMemcpyHostToDevice, c->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(tmp + n, u, 3 * n * sizeof(double), cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "set_fields copy");
        drho = tmp;
        du = tmp + n;
    }
    cudaError_t e = launch_init_equilibrium(c->prec, c->fA, c->L, drho, du, c->fields, c->stream);
    c->launches++;
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_watch, 0, 2 * sizeof(double), c->stream);  // new reference mass
    if (e != cudaSuccess) return cuda_fail(c, e, "init kernel");
    if (!on_device) {
        e = cudaStreamSynchronize(c->stream);  // the host buffers may be freed after return
        if (e != cudaSuccess) return cuda_fail(c, e, "set_fields sync");
    }
    return LBIB_OK;
}

int lbib_set_populations(void *h, const double *f, int on_device) {
    Ctx *c = as_ctx(h);
    if (!c || !f) return LBIB_EINVAL;
    const size_t n = (size_t)c->L.ncell * Q;
    const double *df = f;
    if (!on_device) {
        double *tmp = get_scratch(c, n * sizeof(double));
        if (!tmp) return fail(c, LBIB_ENOMEM, "scratch allocation failed");
        cudaError_t e = cudaMemcpyAsync(tmp, f, n * sizeof(double), cudaMemcpyHostToDevice, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "set_populations copy");
        df = tmp;
    }
    cudaError_t e = launch_aos_to_pop(c->prec, df, c->L, c->fA, c->stream);
    c->launches++;
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_watch, 0, 2 * sizeof(double), c->stream);  // new reference mass
    if (e != cudaSuccess) return cuda_fail(c, e, "populations kernel");
    if (!on_device) {
        e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "set_populations sync");
    }
    return LBIB_OK;
}

int lbib_add_body(void *h, const double *verts, int nv, const int *tris, int nt, const lbib_body_params *bp,
                  int *body_id) {
    Ctx *c = as_ctx(h);
    if (!c || !verts || !tris || !bp) return LBIB_EINVAL;
    if (c->err) return c->err;
    if (nv < 4 || nt < 4) return fail(c, LBIB_EINVAL, "a body needs at least 4 vertices and 4 triangles");
    for (int a = 0; a < 3; ++a) {
        const int na = a == 0 ? c->L.nx : a == 1 ? c->L.ny : c->L.nz;
        if (c->L.bc[a] == kWall && na < 5)
            return fail(c, LBIB_EINVAL, "bodies need at least 5 nodes along walled axes");
    }
    for (int i = 0; i < 3 * nt; ++i)
        if (tris[i] < 0 || tris[i] >= nv) return fail(c, LBIB_EINVAL, "triangle index out of range");
    for (int i = 0; i < 3 * nv; ++i)
        if (!std::isfinite(verts[i])) return fail(c, LBIB_EINVAL, "non-finite vertex");
    if (bp->rigid) {
        if (!(bp->density_ratio > 0)) return fail(c, LBIB_EINVAL, "rigid body needs density_ratio > 0");
    } else {
        if (!(bp->thickness > 0) || !(bp->density_ratio > 0) || bp->ks0 < 0 || bp->Eb < 0 || bp->kv < 0 ||
            (bp->Eb > 0 && !(bp->ref_radius > 0)) || (bp->mass_model != 0 && bp->mass_model != 1))
            return fail(c, LBIB_EINVAL, "invalid membrane parameters");
    }
    DevBody b;
    b.nv = nv;
    b.nt = nt;
    b.rigid = bp->rigid ? 1 : 0;
    b.p = *bp;
    // hinges: one per undirected edge a<b, T1 holds a->b, T2 holds b->a.
    // The directed edges leaving each vertex, in triangle order (a CSR table
    // built by counting); an edge's twin is found among the few edges
    // leaving its end vertex.
    std::vector<int> out_ptr(nv + 1, 0);
    for (int k = 0; k < 3 * nt; ++k) out_ptr[tris[k] + 1]++;
    for (int v = 0; v < nv; ++v) out_ptr[v + 1] += out_ptr[v];
    std::vector<int> out_edge(3 * (size_t)nt);  // directed edge id 3 t + s (from corner s of t to corner s+1)
    {
        std::vector<int> fill(out_ptr.begin(), out_ptr.end() - 1);
        for (int t = 0; t < nt; ++t)
            for (int s = 0; s < 3; ++s) out_edge[fill[tris[3 * t + s]]++] = 3 * t + s;
    }
    auto edge_to = [&](int e) { return tris[3 * (e / 3) + (e % 3 + 1) % 3]; };
    // each vertex's edges sorted by their end vertex: a repeated directed
    // edge shows as two equal neighbours, a twin is found by bisection
    // (O(d log d) for a vertex of degree d, whatever the mesh)
    for (int v = 0; v < nv; ++v) {
        std::sort(out_edge.begin() + out_ptr[v], out_edge.begin() + out_ptr[v + 1],
                  [&](int e, int f) { return edge_to(e) < edge_to(f); });
        for (int p = out_ptr[v] + 1; p < out_ptr[v + 1]; ++p)
            if (edge_to(out_edge[p]) == edge_to(out_edge[p - 1]))
                return fail(c, LBIB_EINVAL, "mesh has a repeated directed edge (not an oriented manifold)");
    }
    std::vector<int4> hinge;
    std::vector<int> htri;
    for (int t = 0; t < nt; ++t)
        for (int s = 0; s < 3; ++s) {
            const int a = tris[3 * t + s], bb = tris[3 * t + (s + 1) % 3];
            // the edge bb -> a
            const auto first = out_edge.begin() + out_ptr[bb], last = out_edge.begin() + out_ptr[bb + 1];
            const auto it = std::lower_bound(first, last, a, [&](int e, int target) { return edge_to(e) < target; });
            if (it == last || edge_to(*it) != a) return fail(c, LBIB_EINVAL, "mesh is not closed (edge without a twin)");
            const int twin = *it;
            if (a < bb) {
                hinge.push_back(make_int4(a, bb, tris[3 * t + (s + 2) % 3], tris[3 * (twin / 3) + (twin % 3 + 2) % 3]));
                htri.push_back(t);
                htri.push_back(twin / 3);
            }
        }
    const int nh = (int)hinge.size();
    b.nh = nh;
    std::vector<double> ks(nh), l0(nh), kb(nh), th0(nh);
    for (int h2 = 0; h2 < nh; ++h2) {
        const int4 H = hinge[h2];
        double r[3];
        v_sub(verts + 3 * H.x, verts + 3 * H.y, r);
        const double l = std::sqrt(v_dot(r, r));
        const double A1 = tri_area(verts, tris + 3 * htri[2 * h2]), A2 = tri_area(verts, tris + 3 * htri[2 * h2 + 1]);
        l0[h2] = l;
        ks[h2] = bp->ks0 * bp->thickness * (A1 + A2) / (l * l);  // Van Gelder, rest values
        kb[h2] = bp->Eb * ks[h2] * bp->ref_radius * bp->ref_radius;
        th0[h2] = dihedral(verts + 3 * H.x, verts + 3 * H.y, verts + 3 * H.z, verts + 3 * H.w);
    }
    double V0 = 0.0, A0 = 0.0;
    for (int t = 0; t < nt; ++t) {
        double cr[3];
        v_cross(verts + 3 * tris[3 * t + 1], verts + 3 * tris[3 * t + 2], cr);
        V0 += v_dot(verts + 3 * tris[3 * t], cr) / 6.0;
        A0 += tri_area(verts, tris + 3 * t);
    }
    if (!(V0 > 0.0)) return fail(c, LBIB_EINVAL, "mesh encloses no positive volume (inward orientation?)");
    b.V0 = V0;
    b.A0 = A0;
    b.mv = bp->mass_model == 1 ? bp->density_ratio * V0 / nv : bp->density_ratio * bp->thickness * A0 / nv;
    for (int v = 0; v < nv; ++v)
        for (int a = 0; a < 3; ++a) b.origin[a] += verts[3 * v + a] / nv;
    // vertex -> (hinge, role) and vertex -> (triangle, corner) lists (CSR by
    // counting; each vertex's entries in increasing hinge or triangle order)
    std::vector<int> vh_ptr(nv + 1, 0), vt_ptr(nv + 1, 0);
    for (int h2 = 0; h2 < nh; ++h2) {
        vh_ptr[hinge[h2].x + 1]++;
        vh_ptr[hinge[h2].y + 1]++;
        vh_ptr[hinge[h2].z + 1]++;
        vh_ptr[hinge[h2].w + 1]++;
    }
    for (int k = 0; k < 3 * nt; ++k) vt_ptr[tris[k] + 1]++;
    for (int v = 0; v < nv; ++v) {
        vh_ptr[v + 1] += vh_ptr[v];
        vt_ptr[v + 1] += vt_ptr[v];
    }
    std::vector<int> vh_list((size_t)vh_ptr[nv]), vt_list((size_t)vt_ptr[nv]);
    {
        std::vector<int> fh(vh_ptr.begin(), vh_ptr.end() - 1), ft(vt_ptr.begin(), vt_ptr.end() - 1);
        for (int h2 = 0; h2 < nh; ++h2) {
            vh_list[fh[hinge[h2].x]++] = 4 * h2 + 0;
            vh_list[fh[hinge[h2].y]++] = 4 * h2 + 1;
            vh_list[fh[hinge[h2].z]++] = 4 * h2 + 2;
            vh_list[fh[hinge[h2].w]++] = 4 * h2 + 3;
        }
        for (int k = 0; k < 3 * nt; ++k) vt_list[ft[tris[k]]++] = k;
    }
    int rc = 0;
    std::vector<double> X(verts, verts + 3 * (size_t)nv);
    std::vector<int> T(tris, tris + 3 * (size_t)nt);
    for (int k = 0; k < 3; ++k) b.X[k] = upload(c, X, &rc);  // x(t-dt) = x(t) at start
    b.U = upload(c, std::vector<double>(3 * (size_t)nv, 0.0), &rc);
    b.Ub = upload(c, std::vector<double>(3 * (size_t)nv, 0.0), &rc);
    b.Fl = upload(c, std::vector<double>(3 * (size_t)nv, 0.0), &rc);
    const bool cm = bp->centroid_markers != 0;
    const int nm = cm ? nt : nv;  // IB markers: vertices or triangle centroids
    if (cm) {
        b.Uc = upload(c, std::vector<double>(3 * (size_t)nt, 0.0), &rc);
        b.Flc = upload(c, std::vector<double>(3 * (size_t)nt, 0.0), &rc);
    }
    b.phi = dev_alloc(c, c->relem * 27 * (size_t)nm);
    b.node = (int *)dev_alloc(c, sizeof(int) * 27 * (size_t)nm);
    b.tri = upload(c, T, &rc);
    // marker binning: the MLS points (markers; probes at their triangle's
    // centroid) ordered by the Morton code of their nearest node
    // floor(X + 1/2), so that a block's points share support nodes
    {
        auto morton = [](int x, int y, int z) {
            uint64_t code = 0;
            for (int bit = 0; bit < 10; ++bit)
                code |= (uint64_t)((x >> bit) & 1) << (3 * bit) | (uint64_t)((y >> bit) & 1) << (3 * bit + 1) |
                        (uint64_t)((z >> bit) & 1) << (3 * bit + 2);
            return code;
        };
        auto cell = [&](const double *P) {
            int q[3];
            for (int a = 0; a < 3; ++a) {
                long long k = (long long)std::floor(P[a] + 0.5);
                q[a] = (int)(k < 0 ? 0 : k & 1023);
            }
            return morton(q[0], q[1], q[2]);
        };
        const int npts = nm + 2 * nt;
        std::vector<std::pair<uint64_t, int>> keyed(npts);
        for (int t = 0; t < nt; ++t) {
            double cen[3];
            for (int a = 0; a < 3; ++a)
                cen[a] = (verts[3 * tris[3 * t] + a] + verts[3 * tris[3 * t + 1] + a] + verts[3 * tris[3 * t + 2] + a]) /
                         3.0;
            const uint64_t k = cell(cen);
            if (cm) keyed[t] = {k, t};
            keyed[nm + 2 * t] = {k, nm + 2 * t};
            keyed[nm + 2 * t + 1] = {k, nm + 2 * t + 1};
        }
        if (!cm)
            for (int v = 0; v < nv; ++v) keyed[v] = {cell(&verts[3 * v]), v};
        std::stable_sort(keyed.begin(), keyed.end(),
                         [](const std::pair<uint64_t, int> &a, const std::pair<uint64_t, int> &b) {
                             return a.first < b.first;
                         });
        std::vector<int> perm(npts);
        for (int k = 0; k < npts; ++k) perm[k] = keyed[k].second;
        b.perm = upload(c, perm, &rc);
    }
    b.tri_geo = dev_alloc(c, c->relem * 8 * (size_t)nt);
    b.tri_vol = (double *)dev_alloc(c, sizeof(double) * (size_t)nt);
    b.probe = dev_alloc(c, c->relem * 8 * (size_t)nt);
    b.vh_ptr = upload(c, vh_ptr, &rc);
    b.vh_list = upload(c, vh_list, &rc);
    b.vt_ptr = upload(c, vt_ptr, &rc);
    b.vt_list = upload(c, vt_list, &rc);
    b.hinge = upload(c, hinge, &rc);
    b.ks = upload_r(c, ks, &rc);
    b.l0 = upload_r(c, l0, &rc);
    b.kb = upload_r(c, kb, &rc);
    b.theta0 = upload_r(c, th0, &rc);
    {
        std::vector<double> xr(3 * (size_t)nv);
        for (int v = 0; v < nv; ++v)
            for (int a = 0; a < 3; ++a) xr[3 * v + a] = verts[3 * v + a] - b.origin[a];
        b.Xrel[0] = upload_r(c, xr, &rc);
        b.Xrel[1] = upload_r(c, xr, &rc);
        if (!b.rigid && c->relem == 4) {
            // the membrane's edge vectors are formed as (hi_j - hi_i) + (lo_j -
            // lo_i): FP32 relative precision of the edge, not of the coordinate
            std::vector<float> lo(xr.size());
            for (size_t k = 0; k < xr.size(); ++k) lo[k] = (float)(xr[k] - (double)(float)xr[k]);
            b.Xlo[0] = static_cast<float *>(upload(c, lo, &rc));
            b.Xlo[1] = static_cast<float *>(upload(c, lo, &rc));
        }
    }
    if (b.rigid) {
        double V, cen[3], I[9];
        mass_props(verts, nt, tris, &V, cen, I);
        std::vector<double> Xb(3 * (size_t)nv), st(RigidState::SIZE, 0.0);
        for (int v = 0; v < nv; ++v)
            for (int a = 0; a < 3; ++a) Xb[3 * v + a] = verts[3 * v + a] - cen[a];
        const double rs = bp->density_ratio;
        for (int a = 0; a < 3; ++a) {
            st[RigidState::XC + a] = cen[a];
            st[RigidState::XC_OLD + a] = cen[a];
            st[RigidState::U + a] = st[RigidState::UP + a] = bp->u0[a];
            st[RigidState::W + a] = st[RigidState::WP + a] = bp->omega0[a];
            st[RigidState::GRAV + a] = bp->gravity[a];
        }
        st[RigidState::Q4] = 1.0;
        st[RigidState::ROT] = st[RigidState::ROT + 4] = st[RigidState::ROT + 8] = 1.0;
        for (int k = 0; k < 9; ++k) st[RigidState::IB + k] = rs * I[k];
        {
            // body-frame inverse inertia (I_world^-1 = R I_b^-1 R^T)
            const double *M = st.data() + RigidState::IB;
            const double det = M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) +
                               M[2] * (M[3] * M[7] - M[4] * M[6]);
            if (!(det > 0.0)) return fail(c, LBIB_EINVAL, "rigid body with a singular inertia tensor");
            double *Mi = st.data() + RigidState::IBINV;
            Mi[0] = (M[4] * M[8] - M[5] * M[7]) / det;
            Mi[1] = (M[2] * M[7] - M[1] * M[8]) / det;
            Mi[2] = (M[1] * M[5] - M[2] * M[4]) / det;
            Mi[3] = (M[5] * M[6] - M[3] * M[8]) / det;
            Mi[4] = (M[0] * M[8] - M[2] * M[6]) / det;
            Mi[5] = (M[2] * M[3] - M[0] * M[5]) / det;
            Mi[6] = (M[3] * M[7] - M[4] * M[6]) / det;
            Mi[7] = (M[1] * M[6] - M[0] * M[7]) / det;
            Mi[8] = (M[0] * M[4] - M[1] * M[3]) / det;
        }
        st[RigidState::MASS] = rs * V;
        st[RigidState::INVM] = 1.0 / (rs * V);
        st[RigidState::VOL] = V;
        st[RigidState::DENS] = rs;
        b.Xbody = upload(c, Xb, &rc);
        b.rstate = upload(c, st, &rc);
    }
    {
        // node box of the supports of the initial markers (kept current by the
        // update kernels from then on)
        std::vector<int> box = {0x7fffffff, 0x7fffffff, 0x7fffffff, (int)0x80000000, (int)0x80000000,
                                (int)0x80000000};
        for (int v = 0; v < nv; ++v)
            for (int a = 0; a < 3; ++a) {
                const int cc = (int)std::floor(verts[3 * v + a]);
                box[a] = std::min(box[a], cc - 3);
                box[3 + a] = std::max(box[3 + a], cc + 4);
            }
        b.bbox[0] = upload(c, box, &rc);
        b.bbox[1] = upload(c, box, &rc);
        BodyView tmp{};
        tmp.nv = nv;
        tmp.nt = nt;
        tmp.nm = nm;
        // partial sums: one per MLS block (membrane volume) or six per
        // force block (rigid force and moment)
        b.nvol_part = std::max(mls_blocks(tmp), 6 * ((nt + 255) / 256));
        b.vol_part = upload(c, std::vector<double>((size_t)b.nvol_part, 0.0), &rc);
        b.vol_sum = upload(c, std::vector<double>(1, 6.0 * V0), &rc);
        b.vol_count = upload(c, std::vector<unsigned int>(1, 0u), &rc);
        // per (vertex, hinge) entry: the hinge's vertices and parameters
        std::vector<int4> hv(vh_list.size());
        std::vector<double> hp(4 * vh_list.size());
        for (size_t q = 0; q < vh_list.size(); ++q) {
            const int h2 = vh_list[q] >> 2;
            hv[q] = hinge[h2];
            hp[4 * q] = ks[h2];
            hp[4 * q + 1] = l0[h2];
            hp[4 * q + 2] = kb[h2];
            hp[4 * q + 3] = th0[h2];
        }
        b.vh_verts = upload(c, hv, &rc);
        b.vh_par = upload_r(c, hp, &rc);
    }
    if (rc || !b.phi || !b.node || !b.tri_geo || !b.tri_vol || !b.probe) {
        c->err = rc ? rc : LBIB_ENOMEM;
        return fail(c, c->err, "body allocation or upload failed");
    }
    cudaError_t e = cudaStreamSynchronize(c->stream);  // host vectors are released on return
    if (e != cudaSuccess) return cuda_fail(c, e, "add_body upload");
    invalidate_graphs(c);
    c->bodies.push_back(b);
    if (body_id) *body_id = (int)c->bodies.size() - 1;
    return LBIB_OK;
}

}  // extern "C"

namespace {

// Enqueues one step on the two step streams (the caller forks them from,
// and joins them into, an origin stream).  With one body, the nodes
// outside its support box do not depend on the IB work of the step: they
// are swept on the low-priority stream concurrently with the IB kernels
// (high priority, so the block scheduler serves them first), and the box is
// swept after the spreading.  ev (6 events or nullptr) receives the stage
// timestamps; `external` records them as graph nodes during capture.
// Advances the host-side buffer rotation but not the step count.
int enqueue_step(Ctx *c, bool store_fields, cudaEvent_t *ev, bool external, int parity) {
    const bool split = c->bodies.size() == 1 && c->split_sweep;
    cudaStream_t hi = c->s_hi, lo = c->s_lo;
    auto rec = [&](int k, cudaStream_t st) {
        if (ev) cudaEventRecordWithFlags(ev[k], st, external ? cudaEventRecordExternal : cudaEventRecordDefault);
    };
    rec(0, hi);
    void *fields = store_fields ? c->fields : nullptr;
    const int *box = split ? c->bodies[0].bbox[c->bodies[0].bcur] : nullptr;
    uint32_t *stamp = c->bodies.empty() ? nullptr : c->stamp;
    if (split) {  // far field on the low-priority stream; it never carries IB force
        rec(4, lo);
        cudaError_t e = launch_sweep(c->prec, c->fA, c->fB, c->force, nullptr, c->d_step, c->L, fields, 1, box,
                                     c->d_sr, parity, c->nsm, lo);
        c->launches++;
        if (e != cudaSuccess) return cuda_fail(c, e, "sweep kernel (outside the body box)");
        rec(5, lo);
        cudaEventRecord(c->ev_far, lo);
    }
    // IB front: support-region moments + MLS at markers and probes
    for (size_t k = 0; k < c->bodies.size(); ++k) {
        const BodyView v = make_view(c, c->bodies[k]);
        cudaError_t e = launch_ib_front(c->prec, c->fA, c->L, v, c->mom, c->nsm, c->d_err,
                                        k == 0 ? c->d_step : nullptr, c->ib_per_sm * c->nsm, hi);
        c->launches += 2;
        if (e != cudaSuccess) return cuda_fail(c, e, "MLS kernels");
    }
    rec(1, hi);
    // structure update and spreading
    for (auto &b : c->bodies) {
        const BodyView v = make_view(c, b);
        cudaError_t e;
        if (b.rigid) {
            e = launch_rigid(c->prec, c->L, v, c->force, c->stamp, c->d_step, c->ib_per_sm * c->nsm, hi);
            c->launches += 2 + v.centroid;
        } else {
            e = launch_membrane(c->prec, c->L, v, c->force, c->stamp, c->d_step, c->ib_per_sm * c->nsm, hi);
            c->launches += 1 + v.centroid;
        }
        if (e != cudaSuccess) return cuda_fail(c, e, "structure kernel");
    }
    rec(2, hi);
    cudaError_t e = launch_sweep(c->prec, c->fA, c->fB, c->force, stamp, c->d_step, c->L, fields, split ? 2 : 0,
                                 box, c->d_sr, parity, c->nsm, hi);
    c->launches++;
    if (e != cudaSuccess) return cuda_fail(c, e, "sweep kernel");
    rec(3, hi);
    if (split) {
        // the next step reads what both sweeps wrote and overwrites what
        // this step's IB work and box sweep read
        cudaStreamWaitEvent(hi, c->ev_far, 0);
        cudaEventRecord(c->ev_near, hi);
        cudaStreamWaitEvent(lo, c->ev_near, 0);
    } else {
        rec(4, hi);
        rec(5, hi);
    }
    std::swap(c->fA, c->fB);
    for (auto &b : c->bodies) {
        b.cur = (b.cur + 1) % 3;
        b.bcur ^= 1;
    }
    return LBIB_OK;
}

// Adds the stage times of one step's six events.
void accumulate_profile(Ctx *c, const cudaEvent_t *ev) {
    float t01 = 0.f, t12 = 0.f, t23 = 0.f, t45 = 0.f, t03 = 0.f, t05 = 0.f;
    cudaEventElapsedTime(&t01, ev[0], ev[1]);
    cudaEventElapsedTime(&t12, ev[1], ev[2]);
    cudaEventElapsedTime(&t23, ev[2], ev[3]);
    cudaEventElapsedTime(&t45, ev[4], ev[5]);
    cudaEventElapsedTime(&t03, ev[0], ev[3]);
    cudaEventElapsedTime(&t05, ev[0], ev[5]);
    c->prof_acc[0] += t01;
    c->prof_acc[1] += t12;
    c->prof_acc[2] += t23 + t45;
    c->prof_acc[3] += t03 > t05 ? t03 : t05;
    c->prof_n++;
}

void harvest_graph_events(Ctx *c, int k) {
    if (!c->gev_pending[k]) return;
    cudaEventSynchronize(c->gev[k][3]);
    cudaEventSynchronize(c->gev[k][5]);
    accumulate_profile(c, c->gev[k]);
    c->gev_pending[k] = false;
}

void invalidate_graphs(Ctx *c) {
    for (int k = 0; k < 6; ++k) {
        harvest_graph_events(c, k);
        if (c->gexec[k]) cudaGraphExecDestroy(c->gexec[k]);
        c->gexec[k] = nullptr;
    }
    c->graphs_valid = false;
}

// Captures one step per phase of the buffer rotation (six steps return the
// rotation to where it started) as CUDA graphs on the capture stream.
int build_graphs(Ctx *c) {
    invalidate_graphs(c);
    for (int k = 0; k < 6; ++k) {
        cudaError_t e = cudaStreamBeginCapture(c->s_cap, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) return cuda_fail(c, e, "graph capture");
        cudaEventRecord(c->ev_fork, c->s_cap);
        cudaStreamWaitEvent(c->s_hi, c->ev_fork, 0);
        cudaStreamWaitEvent(c->s_lo, c->ev_fork, 0);
        const long long launches = c->launches;
        int rc = enqueue_step(c, false, c->profile ? c->gev[k] : nullptr, true, (int)((c->steps + k) & 1));
        c->launches = launches;
        cudaEventRecord(c->ev_join, c->s_hi);
        cudaStreamWaitEvent(c->s_cap, c->ev_join, 0);
        cudaGraph_t g = nullptr;
        e = cudaStreamEndCapture(c->s_cap, &g);
        if (rc) {
            if (g) cudaGraphDestroy(g);
            return rc;
        }
        if (e != cudaSuccess) return cuda_fail(c, e, "graph capture end");
        // kernel nodes keep the priority of the stream they were captured from
        e = cudaGraphInstantiateWithFlags(&c->gexec[k], g, cudaGraphInstantiateFlagUseNodePriority);
        cudaGraphDestroy(g);
        if (e != cudaSuccess) return cuda_fail(c, e, "graph instantiate");
    }
    c->graph_origin = c->steps;
    c->graphs_timed = c->profile;
    c->graphs_valid = true;
    return LBIB_OK;
}

// launches per step (for the counters when a graph runs the step)
long long launches_per_step(const Ctx *c) {
    long long n = 1 + (c->bodies.size() == 1 && c->split_sweep ? 1 : 0);
    for (auto &b : c->bodies) n += 2 + (b.rigid ? 2 : 1);
    return n;
}

// nsteps steps; with fields_every = 0 the fields are stored on the last of
// them when end_of_call (the last step of a public call)
int step_steps(Ctx *c, int nsteps, bool end_of_call) {
    if (!c) return LBIB_EINVAL;
    if (c->err) return c->err;
    if (nsteps < 0) return fail(c, LBIB_EINVAL, "nsteps < 0");
    if (nsteps == 0) return LBIB_OK;
    for (int it = 0; it < nsteps; ++it) {
        if (!c->bodies.empty() && ++c->step_host == 0xFFFFFFFFu) {
            // before the counter wraps: clear the tile flags and restart it
            cudaError_t e = cudaMemsetAsync(c->stamp, 0, sizeof(uint32_t) * (size_t)c->ntiles, c->stream);
            if (e == cudaSuccess) e = cudaMemsetAsync(c->d_step, 0, sizeof(uint32_t), c->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(c->d_sr, 0, 2 * sizeof(uint32_t), c->stream);
    if (e == cudaSuccess)
        e = cudaMemsetAsync(c->d_tot, 0, sizeof(double) * (size_t)totals_scratch_doubles(), c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "step counter reset");
            c->step_host = 1;
        }
        const bool store = c->fields_every == 0 ? (end_of_call && it == nsteps - 1)
                                                : (c->fields_every > 0 && (c->steps + 1) % c->fields_every == 0);
        if (c->use_graphs && !store) {
            if (!c->graphs_valid || c->graphs_timed != c->profile) {
                int rc = build_graphs(c);
                if (rc) return rc;
            }
            const int k = (int)(((c->steps - c->graph_origin) % 6 + 6) % 6);
            harvest_graph_events(c, k);
            cudaError_t e = cudaGraphLaunch(c->gexec[k], c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "graph launch");
            if (c->profile) c->gev_pending[k] = true;
            // the graph performs the buffer rotation of its step: mirror it
            std::swap(c->fA, c->fB);
            for (auto &b : c->bodies) {
                b.cur = (b.cur + 1) % 3;
                b.bcur ^= 1;
            }
            c->launches += launches_per_step(c);
        } else {
            cudaEvent_t *ev = nullptr;
            if (c->profile) {
                if (c->nev + 6 > c->events.size())
                    for (int k = 0; k < 6; ++k) {
                        cudaEvent_t x;
                        if (cudaEventCreate(&x) != cudaSuccess) return cuda_fail(c, cudaGetLastError(), "event");
                        c->events.push_back(x);
                    }
                ev = &c->events[c->nev];
                c->nev += 6;
            }
            cudaEventRecord(c->ev_fork, c->stream);
            cudaStreamWaitEvent(c->s_hi, c->ev_fork, 0);
            cudaStreamWaitEvent(c->s_lo, c->ev_fork, 0);
            int rc = enqueue_step(c, store, ev, false, (int)(c->steps & 1));
            if (rc) return rc;
            cudaEventRecord(c->ev_join, c->s_hi);
            cudaStreamWaitEvent(c->stream, c->ev_join, 0);
        }
        c->steps++;
        if (c->watch_every > 0 && c->steps % c->watch_every == 0) {
            int rc = enqueue_watch(c, c->stream);
            if (rc) return rc;
        }
    }
    return LBIB_OK;
}

}  // namespace

extern "C" {

int lbib_step(void *h, int nsteps) { return step_steps(as_ctx(h), nsteps, true); }

int lbib_set_watchdog(void *h, int every, double mass_tol) {
    Ctx *c = as_ctx(h);
    if (!c) return LBIB_EINVAL;
    if (every < 0 || !(mass_tol > 0.0)) return fail(c, LBIB_EINVAL, "watchdog: every >= 0 and mass_tol > 0");
    c->watch_every = every;
    c->watch_tol = mass_tol;
    return LBIB_OK;
}

int lbib_check(void *h) {
    Ctx *c = as_ctx(h);
    if (!c) return LBIB_EINVAL;
    if (c->err) return c->err;
    int rc = enqueue_watch(c, c->stream);
    if (rc) return rc;
    return sync_ctx(c);
}

int lbib_sync(void *h) {
    Ctx *c = as_ctx(h);
    if (!c) return LBIB_EINVAL;
    return sync_ctx(c);
}

int lbib_get_fields(void *h, double *rho, double *u, int on_device) {
    Ctx *c = as_ctx(h);
    if (!c) return LBIB_EINVAL;
    int rc = sync_ctx(c);
    if (rc && !readable_error(rc)) return rc;
    const size_t n = (size_t)c->L.ncell;
    double *drho = rho, *du = u;
    if (!on_device) {
        double *tmp = get_scratch(c, 4 * n * sizeof(double));
        if (!tmp) return fail(c, LBIB_ENOMEM, "scratch allocation failed");
        drho = rho ? tmp : nullptr;
        du = u ? tmp + n : nullptr;
    }
    cudaError_t e = launch_fields_out(c->prec, c->fields, c->L, drho, du, c->stream);
    c->launches++;
    if (e != cudaSuccess) return cuda_fail(c, e, "fields kernel");
    if (!on_device) {
        if (rho) e = cudaMemcpyAsync(rho, drho, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess && u) e = cudaMemcpyAsync(u, du, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "fields copy");
    }
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "fields sync");
    return rc;
}

int lbib_get_totals(void *h, double *out) {
    Ctx *c = as_ctx(h);
    if (!c || !out) return LBIB_EINVAL;
    int rc = sync_ctx(c);
    if (rc && !readable_error(rc)) return rc;
    const int n = totals_scratch_doubles();
    double *part = c->d_tot, *res = c->d_tot + (n - 8);
    unsigned int *count = reinterpret_cast<unsigned int *>(c->d_tot + (n - 4));
    cudaError_t e = launch_totals(c->prec, c->fA, c->L, part, count, res, c->stream);
    c->launches++;
    if (e == cudaSuccess) e = cudaMemcpyAsync(out, res, 4 * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "totals");
    return rc;
}

int lbib_get_populations(void *h, double *f, int on_device) {
    Ctx *c = as_ctx(h);
    if (!c || !f) return LBIB_EINVAL;
    int rc = sync_ctx(c);
    if (rc && !readable_error(rc)) return rc;
    const size_t n = (size_t)c->L.ncell * Q;
    double *df = f;
    if (!on_device) {
        df = get_scratch(c, n * sizeof(double));
        if (!df) return fail(c, LBIB_ENOMEM, "scratch allocation failed");
    }
    cudaError_t e = launch_pop_to_aos(c->prec, c->fA, c->L, df, c->stream);
    c->launches++;
    if (e != cudaSuccess) return cuda_fail(c, e, "populations kernel");
    if (!on_device) {
        e = cudaMemcpyAsync(f, df, n * sizeof(double), cudaMemcpyDeviceToHost, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "populations copy");
    }
    e = cudaStreamSynchronize(c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "populations sync");
    return rc;
}

int lbib_get_markers_async(void *h, int body, double *X, double *V, double *F) {
    Ctx *c = as_ctx(h);
    if (!c) return LBIB_EINVAL;
    if (body < 0 || body >= (int)c->bodies.size()) return fail(c, LBIB_EINVAL, "no such body");
    if (c->err && !readable_error(c->err)) return c->err;
    DevBody &b = c->bodies[body];
    const size_t bytes = 3 * (size_t)b.nv * sizeof(double);
    cudaError_t e = cudaSuccess;
    if (X) e = cudaMemcpyAsync(X, b.X[b.cur], bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && V) e = cudaMemcpyAsync(V, b.Ub, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && F) e = cudaMemcpyAsync(F, b.Fl, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "markers copy");
    return LBIB_OK;
}

// Step k's markers into slot k of the staging planes (X, U_b, F_l).
__global__ void k_stage_markers(const double *__restrict__ X, const double *__restrict__ Ub,
                                const double *__restrict__ Fl, double *__restrict__ dst, long long n3,
                                long long plane, int slot) {
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n3; i += (long long)gridDim.x * blockDim.x) {
        if (X) dst[slot * n3 + i] = X[i];
        if (Ub) dst[plane + slot * n3 + i] = Ub[i];
        if (Fl) dst[2 * plane + slot * n3 + i] = Fl[i];
    }
}

int lbib_step_markers(void *h, int nsteps, int body, double *X, double *V, double *F) {
    Ctx *c = as_ctx(h);
    if (!c || nsteps < 0) return LBIB_EINVAL;
    if (body < 0 || body >= (int)c->bodies.size()) return fail(c, LBIB_EINVAL, "no such body");
    if (nsteps == 0) return LBIB_OK;
    if (c->err && !readable_error(c->err)) return c->err;
    const size_t n3 = 3 * (size_t)c->bodies[body].nv;
    const size_t plane = n3 * (size_t)nsteps, need = 3 * plane * sizeof(double);
    if (need > c->mstage_bytes) {
        // a larger staging buffer; the old one may still feed queued copies
        if (c->mstage) {
            cudaError_t e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "marker staging");
            dev_free_one(c, c->mstage);
            c->mstage = nullptr;
            c->mstage_bytes = 0;
        }
        c->mstage = static_cast<double *>(dev_alloc(c, need));
        if (!c->mstage) return fail(c, LBIB_ENOMEM, "marker staging buffer of %zu bytes", need);
        c->mstage_bytes = need;
    }
    // each step's markers go to the staging planes on the device (one small
    // kernel behind the step); the host copies follow the last step, one
    // per requested array
    const int blocks = (int)std::min<size_t>((n3 + 255) / 256, 1024);
    for (int k = 0; k < nsteps; ++k) {
        // one step at a time, the fields stored as lbib_step(h, nsteps) would
        int rc = step_steps(c, 1, k == nsteps - 1);
        if (rc) return rc;
        DevBody &b = c->bodies[body];
        k_stage_markers<<<blocks, 256, 0, c->stream>>>(X ? b.X[b.cur] : nullptr, V ? b.Ub : nullptr,
                                                       F ? b.Fl : nullptr, c->mstage, (long long)n3,
                                                       (long long)plane, k);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(c, e, "marker staging");
        c->launches++;
    }
    const size_t bytes = plane * sizeof(double);
    cudaError_t e = cudaSuccess;
    if (X) e = cudaMemcpyAsync(X, c->mstage, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && V) e = cudaMemcpyAsync(V, c->mstage + plane, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e == cudaSuccess && F) e = cudaMemcpyAsync(F, c->mstage + 2 * plane, bytes, cudaMemcpyDeviceToHost, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "markers copy");
    return LBIB_OK;
}

int lbib_get_markers(void *h, int body, double *X, double *V, double *F) {
    // the copies and the device error word in one round trip
    int rc = lbib_get_markers_async(h, body, X, V, F);
    if (rc) return rc;
    return sync_ctx(as_ctx(h));
}

int lbib_get_body(void *h, int body, lbib_body_state *out) {
    Ctx *c = as_ctx(h);
    if (!c || !out) return LBIB_EINVAL;
    if (body < 0 || body >= (int)c->bodies.size()) return fail(c, LBIB_EINVAL, "no such body");
    DevBody &b = c->bodies[body];
    std::vector<double> X(3 * (size_t)b.nv), Ub(3 * (size_t)b.nv);
    int rc = lbib_get_markers(h, body, X.data(), Ub.data(), nullptr);
    if (rc && !readable_error(rc)) return rc;
    std::memset(out, 0, sizeof(*out));
    if (b.rigid) {
        double st[RigidState::SIZE];
        cudaError_t e = cudaMemcpy(st, b.rstate, sizeof(st), cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(c, e, "body state copy");
        for (int a = 0; a < 3; ++a) {
            out->xc[a] = st[RigidState::XC + a];
            out->u[a] = st[RigidState::U + a];
            out->omega[a] = st[RigidState::W + a];
        }
        for (int k = 0; k < 4; ++k) out->q[k] = st[RigidState::Q4 + k];
    } else {
        for (int v = 0; v < b.nv; ++v)
            for (int a = 0; a < 3; ++a) {
                out->xc[a] += X[3 * v + a] / b.nv;
                out->u[a] += Ub[3 * v + a] / b.nv;
            }
        out->q[0] = 1.0;
    }
    std::vector<int> T(3 * (size_t)b.nt);
    cudaError_t e = cudaMemcpy(T.data(), b.tri, T.size() * sizeof(int), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(c, e, "triangles copy");
    double V = 0, A = 0;
    for (int t = 0; t < b.nt; ++t) {
        double cr[3];
        v_cross(&X[3 * T[3 * t + 1]], &X[3 * T[3 * t + 2]], cr);
        V += v_dot(&X[3 * T[3 * t]], cr) / 6.0;
        A += tri_area(X.data(), &T[3 * t]);
    }
    out->volume = V;
    out->area = A;
    return rc;
}

int lbib_counters(void *h, long long *steps, long long *launches) {
    Ctx *c = as_ctx(h);
    if (!c) return LBIB_EINVAL;
    if (steps) *steps = c->steps;
    if (launches) *launches = c->launches;
    return LBIB_OK;
}

int lbib_profile(void *h, int enable) {
    Ctx *c = as_ctx(h);
    if (!c) return LBIB_EINVAL;
    if (!enable)
        for (int k = 0; k < 6; ++k) c->gev_pending[k] = false;
    c->profile = enable != 0;
    return LBIB_OK;
}

int lbib_get_profile(void *h, double *ms, long long *nsteps) {
    Ctx *c = as_ctx(h);
    if (!c || !ms) return LBIB_EINVAL;
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->s_hi);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->s_lo);
    if (e != cudaSuccess) return cuda_fail(c, e, "profile sync");
    for (size_t k = 0; k + 6 <= c->nev; k += 6) accumulate_profile(c, &c->events[k]);
    for (int k = 0; k < 6; ++k) harvest_graph_events(c, k);
    for (int j = 0; j < 4; ++j) ms[j] = c->prof_acc[j];
    if (nsteps) *nsteps = c->prof_n;
    c->nev = 0;
    for (int j = 0; j < 4; ++j) c->prof_acc[j] = 0.0;
    c->prof_n = 0;
    return LBIB_OK;
}

int lbib_set_graphs(void *h, int enable) {
    Ctx *c = as_ctx(h);
    if (!c) return LBIB_EINVAL;
    c->use_graphs = enable != 0;
    return LBIB_OK;
}

int lbib_autotune(void *h, int steps, int *choice) {
    Ctx *c = as_ctx(h);
    if (!c || steps < 1) return LBIB_EINVAL;
    if (c->err) return c->err;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return cuda_fail(c, cudaGetLastError(), "autotune events");
    // one untimed step (it captures the step graphs of the configuration),
    // then the best of two timed runs of `steps` steps
    auto trial = [&](float *ms) -> int {
        int rc = lbib_step(h, 1);
        if (rc) return rc;
        *ms = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
            cudaEventRecord(e0, c->stream);
            if ((rc = lbib_step(h, steps))) return rc;
            cudaEventRecord(e1, c->stream);
            cudaError_t e = cudaEventSynchronize(e1);
            if (e != cudaSuccess) return cuda_fail(c, e, "autotune sync");
            float t = 0.f;
            cudaEventElapsedTime(&t, e0, e1);
            if (t < *ms) *ms = t;
        }
        return sync_ctx(c);
    };
    // sweep launch shapes: the row-tile kernel (where it applies), whole
    // x-rows of the one-node kernel, then fixed 2D shapes
    const int shapes[][3] = {{0, 0, 0}, {0, 0, 1}, {32, 8, 0}, {64, 4, 0}, {128, 2, 0}, {256, 1, 0}, {32, 4, 0},
                             {64, 2, 0}};
    const int esz = c->prec == LBIB_FP64 ? 8 : c->prec == LBIB_FP32 ? 4 : 2;
    const bool vec_ok = (c->L.nx & 3) == 0 && (c->L.nx * esz) % 16 == 0 &&
                        19LL * std::max(1, std::min(256 / c->L.nx, c->L.ny)) * c->L.nx * esz <= 160 * 1024 &&
                        c->L.nx <= 512;
    const bool saved_split = c->split_sweep;
    c->split_sweep = false;
    float best = 1e30f;
    int best_shape = 0, rc = 0;
    for (int k = 0; k < (int)(sizeof(shapes) / sizeof(shapes[0])); ++k) {
        if (shapes[k][2] && !vec_ok) continue;
        if (shapes[k][0] > 0 && shapes[k][0] > (c->L.nx + 31) / 32 * 32) continue;
        c->L.sweep_bx = shapes[k][0];
        c->L.sweep_by = shapes[k][1];
        c->L.sweep_vec = shapes[k][2];
        invalidate_graphs(c);
        float ms = 0.f;
        if ((rc = trial(&ms))) break;
        if (ms < best) {
            best = ms;
            best_shape = k;
        }
    }
    c->L.sweep_bx = shapes[best_shape][0];
    c->L.sweep_by = shapes[best_shape][1];
    c->L.sweep_vec = shapes[best_shape][2];
    invalidate_graphs(c);
    // overlap of the far-field sweep with the IB stage, the far-field sweep
    // on its full grid or on a few resident blocks per SM, the IB kernels on
    // their full grids or on one or two resident blocks per SM
    int overlap = 0, far = 0, ibs = 0;
    const int saved_ibs = c->ib_per_sm;
    c->ib_per_sm = 0;
    if (!rc && c->bodies.size() == 1) {
        c->split_sweep = true;
        for (int fps : {0, 1, 2, 3})
            for (int ib : {0, 1, 2}) {
                if (rc) break;
                float ms = 0.f;
                c->L.far_per_sm = fps;
                c->ib_per_sm = ib;
                invalidate_graphs(c);
                if ((rc = trial(&ms))) break;
                if (ms < best) {
                    best = ms;
                    overlap = 1;
                    far = fps;
                    ibs = ib;
                }
            }
    } else {
        (void)saved_split;
        (void)saved_ibs;
    }
    c->L.far_per_sm = far;
    c->ib_per_sm = ibs;
    c->split_sweep = overlap != 0;
    invalidate_graphs(c);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (choice) {
        choice[0] = c->L.sweep_bx;
        choice[1] = c->L.sweep_by;
        choice[2] = overlap;
        choice[3] = c->L.sweep_vec;
        choice[4] = c->L.far_per_sm;
    }
    return rc;
}

int lbib_set_sweep_config(void *h, int row_tiles, int block_x, int block_y, int far_per_sm) {
    Ctx *c = as_ctx(h);
    if (!c) return LBIB_EINVAL;
    if (row_tiles < 0 || row_tiles > 1 || block_x < 0 || block_y < 0 || (block_x == 0) != (block_y == 0) ||
        block_x * block_y > 1024 || far_per_sm < 0 || far_per_sm > 64)
        return fail(c, LBIB_EINVAL, "bad sweep configuration");
    c->L.sweep_vec = row_tiles;
    c->L.far_per_sm = far_per_sm;
    c->L.sweep_bx = block_x;
    c->L.sweep_by = block_y;
    invalidate_graphs(c);
    return LBIB_OK;
}

int lbib_set_ib_blocks(void *h, int per_sm) {
    Ctx *c = as_ctx(h);
    if (!c) return LBIB_EINVAL;
    if (per_sm < 0 || per_sm > 64) return fail(c, LBIB_EINVAL, "IB blocks per SM must lie in [0, 64]");
    if (c->ib_per_sm != per_sm) invalidate_graphs(c);
    c->ib_per_sm = per_sm;
    return LBIB_OK;
}

int lbib_get_launch_config(void *h, int *cfg) {
    Ctx *c = as_ctx(h);
    if (!c || !cfg) return LBIB_EINVAL;
    cfg[0] = c->L.sweep_bx;
    cfg[1] = c->L.sweep_by;
    cfg[2] = c->split_sweep ? 1 : 0;
    cfg[3] = c->L.sweep_vec;
    cfg[4] = c->L.far_per_sm;
    cfg[5] = c->ib_per_sm;
    return LBIB_OK;
}

int lbib_set_overlap(void *h, int enable) {
    Ctx *c = as_ctx(h);
    if (!c) return LBIB_EINVAL;
    if (c->split_sweep != (enable != 0)) invalidate_graphs(c);
    c->split_sweep = enable != 0;
    return LBIB_OK;
}

int lbib_set_output(void *h, int fields_every) {
    Ctx *c = as_ctx(h);
    if (!c) return LBIB_EINVAL;
    c->fields_every = fields_every;
    return LBIB_OK;
}

int lbib_device_bytes(void *h, size_t *bytes) {
    Ctx *c = as_ctx(h);
    if (!c || !bytes) return LBIB_EINVAL;
    *bytes = c->bytes;
    return LBIB_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Batches: the lattices and bodies of several contexts advanced by common
// launches (one moments, MLS, structure and sweep launch per step for the
// whole batch), optionally replayed six steps at a time from a CUDA graph.
// ---------------------------------------------------------------------------
namespace {

struct Batch {
    std::vector<Ctx *> ctx;
    std::vector<long long> base;      // step count of each context at the last table build
    std::vector<cudaEvent_t> ctx_ev;  // per context: its stream's work before a batch call
    int prec = 1;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    cudaStream_t s_cap = nullptr;  // private capture stream: the batch stream is never in capture mode
    cudaEvent_t done = nullptr;
    // sweep of each lattice as its own launch (the one-lattice kernel with its
    // parameters in the constant bank), spread over side streams
    int sweep_split = 0;
    std::vector<cudaStream_t> side;
    std::vector<cudaEvent_t> side_ev;  // [0] fork, [1..] joins
    std::vector<Lattice> lat_h;        // host copies of the launch tables
    std::vector<LatRef> ref_h;
    std::vector<int> order_h;
    int nsm = 1;
    void *dmem = nullptr;
    BatchTables T{};
    BatchGrid G{};
    long long steps = 0;  // steps since the last table build (phase origin)
    int sweep_threads = 256, order = 0, sweep_cpt = 4;
    cudaGraphExec_t g6 = nullptr;
    long long launches = 0, total_steps = 0;
    std::string msg;
    // persistent mode: the six-step chunks run as one kernel launch over a
    // queue of work items (kp_batch)
    int persistent = 0;
    double wait_s = 2.0;       // bound on each dependency wait of the persistent kernel
    void *pmem = nullptr;      // its item tables and counters
    PersistTables P{};
    unsigned *pctr = nullptr;  // ticket, abort flag and completion counters (zeroed per launch)
    size_t pctr_bytes = 0;
    int pgrid = 0;             // resident blocks of the persistent kernel
};

std::string g_batch_error;

int bfail(Batch *b, int code, const char *what) {
    if (b)
        b->msg = what;
    else
        g_batch_error = what;
    return code;
}

int bcuda(Batch *b, cudaError_t e, const char *what) {
    std::string m = std::string(what) + ": " + cudaGetErrorString(e);
    return bfail(b, LBIB_ECUDA, m.c_str());
}

void batch_free_tables(Batch *b) {
    if (b->g6) cudaGraphExecDestroy(b->g6);
    b->g6 = nullptr;
    if (b->dmem) cudaFree(b->dmem);
    b->dmem = nullptr;
    if (b->pmem) cudaFree(b->pmem);
    b->pmem = nullptr;
    b->pctr = nullptr;
}

// Work items of the persistent kernel's six-step launch, in queue order.
// Per body: support-moment, MLS, membrane, rigid-force, rigid-marker and
// centroid items (each split into the blocks the separate kernels would
// launch); per lattice: sweep tiles of sweep_cells cells.  Each lattice's
// chain of phases (its item kinds in order, step after step) is laid out in
// rounds, lattice l's phase j in round j + offset(l), the offsets spreading
// the lattices (in sweep order) over one step's phases: every stretch of
// the queue mixes some lattices' sweeps with other lattices' IB phases,
// and a phase's items sit a round after the phase they depend on.
// need[l][k]: items of kind k of lattice l per step.
int batch_build_persistent(Batch *b, const std::vector<std::pair<int, int>> &bodies,
                           const std::vector<BodyRef> &body, const std::vector<Lattice> &lat,
                           const std::vector<int> &order) {
    const int nl = (int)lat.size(), nb = (int)bodies.size(), nsteps = 6;
    const int cells = 256 * b->sweep_cpt;
    std::vector<int> body_lat(nb > 0 ? nb : 1, 0);
    std::vector<unsigned> need((size_t)nl * kPKinds, 0u);
    std::vector<std::array<int, kPKinds>> count(nb);  // items per step of each body and kind
    std::vector<std::vector<int>> lat_bodies(nl);
    for (int q = 0; q < nb; ++q) {
        body_lat[q] = bodies[q].first;
        lat_bodies[bodies[q].first].push_back(q);
        const DevBody &d = b->ctx[bodies[q].first]->bodies[bodies[q].second];
        std::array<int, kPKinds> &n = count[q];
        n.fill(0);
        n[kPMom] = std::max(8, d.nv / 16);
        n[kPMls] = mls_blocks(body[q].v);
        n[kPMemb] = d.rigid ? 0 : (d.nv + 7) / 8;
        n[kPRf] = d.rigid ? (d.nt + 255) / 256 : 0;
        n[kPRm] = d.rigid ? (d.nv + 7) / 8 : 0;
        n[kPCen] = d.p.centroid_markers ? (d.nt + 7) / 8 : 0;
        for (int k = kPMom; k < kPSweep; ++k) need[(size_t)bodies[q].first * kPKinds + k] += (unsigned)n[k];
    }
    std::vector<int> tiles(nl);
    for (int l = 0; l < nl; ++l) {
        tiles[l] = (lat[l].ncell + cells - 1) / cells;
        need[(size_t)l * kPKinds + kPSweep] = (unsigned)tiles[l];
    }
    // each lattice's phase kinds, and the rounds
    std::vector<std::vector<int>> kinds(nl);
    int pmax = 1;
    for (int l = 0; l < nl; ++l) {
        for (int k = kPMom; k < kPKinds; ++k)
            if (need[(size_t)l * kPKinds + k]) kinds[l].push_back(k);
        pmax = std::max(pmax, (int)kinds[l].size());
    }
    std::vector<int> offset(nl);
    for (int i = 0; i < nl; ++i) offset[order[i]] = (int)((long long)i * pmax / nl);
    std::vector<int4> items;
    const int rounds = nsteps * pmax + pmax;
    for (int r = 0; r < rounds; ++r)
        for (int i = 0; i < nl; ++i) {
            const int l = order[i], np = (int)kinds[l].size(), j = r - offset[l];
            if (j < 0 || j >= nsteps * np) continue;
            const int st = j / np, k = kinds[l][j % np], tag = k | (st << 8);
            if (k == kPSweep) {
                for (int t = 0; t < tiles[l]; ++t) items.push_back(make_int4(tag, l, t, tiles[l]));
            } else {
                for (int q : lat_bodies[l])
                    for (int vb = 0; vb < count[q][k]; ++vb) items.push_back(make_int4(tag, q, vb, count[q][k]));
            }
        }
    size_t off = 0;
    auto place = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) / 256 * 256;
        return o;
    };
    const size_t o_it = place(sizeof(int4) * items.size()), o_bl = place(sizeof(int) * body_lat.size()),
                 o_nd = place(sizeof(unsigned) * need.size()), o_ct = place(sizeof(unsigned) * (2 + need.size()));
    cudaError_t e = cudaMalloc(&b->pmem, off);
    if (e != cudaSuccess) {
        b->pmem = nullptr;
        return bcuda(b, e, "persistent tables");
    }
    std::vector<unsigned char> host(off, 0);
    std::memcpy(host.data() + o_it, items.data(), sizeof(int4) * items.size());
    std::memcpy(host.data() + o_bl, body_lat.data(), sizeof(int) * body_lat.size());
    std::memcpy(host.data() + o_nd, need.data(), sizeof(unsigned) * need.size());
    e = cudaMemcpy(b->pmem, host.data(), off, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bcuda(b, e, "persistent tables upload");
    unsigned char *d = static_cast<unsigned char *>(b->pmem);
    PersistTables &P = b->P;
    P.nitems = (int)items.size();
    P.nsteps = nsteps;
    P.phase0 = 0;
    P.sweep_cells = cells;
    P.wait_ns = (long long)(b->wait_s * 1e9);
    P.items = reinterpret_cast<const int4 *>(d + o_it);
    P.body_lat = reinterpret_cast<const int *>(d + o_bl);
    P.need = reinterpret_cast<const unsigned *>(d + o_nd);
    b->pctr = reinterpret_cast<unsigned *>(d + o_ct);
    b->pctr_bytes = sizeof(unsigned) * (2 + need.size());
    P.ticket = b->pctr;
    P.abort = b->pctr + 1;
    P.done = b->pctr + 2;
    bool off32 = true;
    for (const Lattice &Li : lat) off32 = off32 && Li.off32;
    const int per_sm = batch_persistent_blocks_per_sm(b->prec, off32);
    if (per_sm < 1) return bfail(b, LBIB_ECUDA, "the persistent kernel does not fit on an SM");
    b->pgrid = per_sm * b->nsm;
    return LBIB_OK;
}

// Builds the launch tables from the contexts' current state (phase 0) and
// the five rotations that follow it.
int batch_build(Batch *b) {
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_free_tables(b);
    const int nl = (int)b->ctx.size();
    std::vector<Lattice> lat(nl);
    std::vector<LatRef> ref(6 * (size_t)nl);
    std::vector<std::pair<int, int>> bodies;  // (context, body)
    for (int i = 0; i < nl; ++i)
        for (int j = 0; j < (int)b->ctx[i]->bodies.size(); ++j) bodies.push_back({i, j});
    const int nb = (int)bodies.size();
    std::vector<BodyRef> body(6 * (size_t)nb);
    for (int i = 0; i < nl; ++i) {
        Ctx *c = b->ctx[i];
        lat[i] = c->L;
        for (int k = 0; k < 6; ++k) {
            LatRef &r = ref[(size_t)k * nl + i];
            r.fin = (k % 2 == 0) ? c->fA : c->fB;
            r.fout = (k % 2 == 0) ? c->fB : c->fA;
            r.force = c->force;
            r.fields = c->fields;
            r.mom = c->mom;
            r.stamp = c->bodies.empty() ? nullptr : c->stamp;
            r.d_step = c->d_step;
            r.err = c->d_err;
            r.sr = c->d_sr;
            r.parity = (int)((c->steps + k) & 1);
        }
    }
    std::vector<int> mom_pre(1, 0), mls_pre(1, 0), memb_id, memb_pre(1, 0), rigid_id, rf_pre(1, 0), rm_pre(1, 0),
        cen_id, cen_pre(1, 0);
    for (int q = 0; q < nb; ++q) {
        Ctx *c = b->ctx[bodies[q].first];
        DevBody &d = c->bodies[bodies[q].second];
        const int cur0 = d.cur, bcur0 = d.bcur;
        for (int k = 0; k < 6; ++k) {
            d.cur = (cur0 + k) % 3;
            d.bcur = bcur0 ^ (k & 1);
            BodyRef &br = body[(size_t)k * nb + q];
            br.v = make_view(c, d);
            br.lat = bodies[q].first;
            br.inc_step = bodies[q].second == 0;
        }
        d.cur = cur0;
        d.bcur = bcur0;
        const BodyView &v = body[q].v;
        mom_pre.push_back(mom_pre.back() + std::max(8, d.nv / 16));
        mls_pre.push_back(mls_pre.back() + mls_blocks(v));
        if (d.rigid) {
            rigid_id.push_back(q);
            rf_pre.push_back(rf_pre.back() + (d.nt + 255) / 256);
            rm_pre.push_back(rm_pre.back() + (d.nv + 7) / 8);
        } else {
            memb_id.push_back(q);
            memb_pre.push_back(memb_pre.back() + (d.nv + 7) / 8);
        }
        if (d.p.centroid_markers) {
            cen_id.push_back(q);
            cen_pre.push_back(cen_pre.back() + (d.nt + 7) / 8);
        }
    }
    // sweep slots: lattices in launch order (0: as given, 1: largest first)
    std::vector<int> order(nl);
    for (int i = 0; i < nl; ++i) order[i] = i;
    if (b->order == 1)
        std::stable_sort(order.begin(), order.end(),
                         [&](int x, int y) { return lat[x].ncell > lat[y].ncell; });
    std::vector<int> sweep_pre(1, 0);
    for (int i = 0; i < nl; ++i)
        sweep_pre.push_back(sweep_pre.back() + (lat[order[i]].ncell + b->sweep_threads * b->sweep_cpt - 1) /
                                                   (b->sweep_threads * b->sweep_cpt));
    // block -> item maps
    auto blocks_of = [](const std::vector<int> &pre) {
        std::vector<int> blk(pre.back() > 0 ? pre.back() : 1, 0);
        for (size_t i = 0; i + 1 < pre.size(); ++i)
            for (int q = pre[i]; q < pre[i + 1]; ++q) blk[q] = (int)i;
        return blk;
    };
    const std::vector<int> sweep_blk = blocks_of(sweep_pre), mom_blk = blocks_of(mom_pre),
                           mls_blk = blocks_of(mls_pre), memb_blk = blocks_of(memb_pre), rf_blk = blocks_of(rf_pre),
                           rm_blk = blocks_of(rm_pre), cen_blk = blocks_of(cen_pre);
    // one device block for all tables
    size_t off = 0;
    auto place = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) / 256 * 256;
        return o;
    };
    const size_t o_lat = place(sizeof(Lattice) * nl), o_ref = place(sizeof(LatRef) * ref.size()),
                 o_body = place(sizeof(BodyRef) * body.size()), o_slat = place(sizeof(int) * nl),
                 o_spre = place(sizeof(int) * sweep_pre.size()), o_mom = place(sizeof(int) * mom_pre.size()),
                 o_mls = place(sizeof(int) * mls_pre.size()), o_mid = place(sizeof(int) * memb_id.size()),
                 o_mpre = place(sizeof(int) * memb_pre.size()), o_rid = place(sizeof(int) * rigid_id.size()),
                 o_rf = place(sizeof(int) * rf_pre.size()), o_rm = place(sizeof(int) * rm_pre.size()),
                 o_bs = place(sizeof(int) * sweep_blk.size()), o_bmo = place(sizeof(int) * mom_blk.size()),
                 o_bml = place(sizeof(int) * mls_blk.size()), o_bme = place(sizeof(int) * memb_blk.size()),
                 o_brf = place(sizeof(int) * rf_blk.size()), o_brm = place(sizeof(int) * rm_blk.size()),
                 o_cid = place(sizeof(int) * cen_id.size()), o_cpre = place(sizeof(int) * cen_pre.size()),
                 o_bce = place(sizeof(int) * cen_blk.size());
    cudaError_t e = cudaMalloc(&b->dmem, off);
    if (e != cudaSuccess) {
        b->dmem = nullptr;
        return bcuda(b, e, "batch tables");
    }
    std::vector<unsigned char> host(off);
    auto put = [&](size_t o, const void *src, size_t bytes) {
        if (bytes) std::memcpy(host.data() + o, src, bytes);
    };
    put(o_lat, lat.data(), sizeof(Lattice) * nl);
    put(o_ref, ref.data(), sizeof(LatRef) * ref.size());
    put(o_body, body.data(), sizeof(BodyRef) * body.size());
    put(o_slat, order.data(), sizeof(int) * nl);
    put(o_spre, sweep_pre.data(), sizeof(int) * sweep_pre.size());
    put(o_mom, mom_pre.data(), sizeof(int) * mom_pre.size());
    put(o_mls, mls_pre.data(), sizeof(int) * mls_pre.size());
    put(o_mid, memb_id.data(), sizeof(int) * memb_id.size());
    put(o_mpre, memb_pre.data(), sizeof(int) * memb_pre.size());
    put(o_rid, rigid_id.data(), sizeof(int) * rigid_id.size());
    put(o_rf, rf_pre.data(), sizeof(int) * rf_pre.size());
    put(o_rm, rm_pre.data(), sizeof(int) * rm_pre.size());
    put(o_bs, sweep_blk.data(), sizeof(int) * sweep_blk.size());
    put(o_bmo, mom_blk.data(), sizeof(int) * mom_blk.size());
    put(o_bml, mls_blk.data(), sizeof(int) * mls_blk.size());
    put(o_bme, memb_blk.data(), sizeof(int) * memb_blk.size());
    put(o_brf, rf_blk.data(), sizeof(int) * rf_blk.size());
    put(o_brm, rm_blk.data(), sizeof(int) * rm_blk.size());
    put(o_cid, cen_id.data(), sizeof(int) * cen_id.size());
    put(o_cpre, cen_pre.data(), sizeof(int) * cen_pre.size());
    put(o_bce, cen_blk.data(), sizeof(int) * cen_blk.size());
    e = cudaMemcpy(b->dmem, host.data(), off, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) return bcuda(b, e, "batch tables upload");
    unsigned char *d = static_cast<unsigned char *>(b->dmem);
    BatchTables &T = b->T;
    T.nl = nl;
    T.nb = nb;
    T.nmemb = (int)memb_id.size();
    T.nrigid = (int)rigid_id.size();
    T.ncen = (int)cen_id.size();
    T.lat = reinterpret_cast<const Lattice *>(d + o_lat);
    T.ref = reinterpret_cast<const LatRef *>(d + o_ref);
    T.body = reinterpret_cast<const BodyRef *>(d + o_body);
    T.sweep_lat = reinterpret_cast<const int *>(d + o_slat);
    T.sweep_pre = reinterpret_cast<const int *>(d + o_spre);
    T.mom_pre = reinterpret_cast<const int *>(d + o_mom);
    T.mls_pre = reinterpret_cast<const int *>(d + o_mls);
    T.memb_id = reinterpret_cast<const int *>(d + o_mid);
    T.memb_pre = reinterpret_cast<const int *>(d + o_mpre);
    T.rigid_id = reinterpret_cast<const int *>(d + o_rid);
    T.rf_pre = reinterpret_cast<const int *>(d + o_rf);
    T.rm_pre = reinterpret_cast<const int *>(d + o_rm);
    T.sweep_blk = reinterpret_cast<const int *>(d + o_bs);
    T.mom_blk = reinterpret_cast<const int *>(d + o_bmo);
    T.mls_blk = reinterpret_cast<const int *>(d + o_bml);
    T.memb_blk = reinterpret_cast<const int *>(d + o_bme);
    T.rf_blk = reinterpret_cast<const int *>(d + o_brf);
    T.rm_blk = reinterpret_cast<const int *>(d + o_brm);
    T.cen_id = reinterpret_cast<const int *>(d + o_cid);
    T.cen_pre = reinterpret_cast<const int *>(d + o_cpre);
    T.cen_blk = reinterpret_cast<const int *>(d + o_bce);
    T.sweep_threads = b->sweep_threads;
    T.sweep_cpt = b->sweep_cpt;
    T.sweep_off32 = 1;
    for (const Lattice &Li : lat) T.sweep_off32 &= Li.off32;
    b->G = BatchGrid{sweep_pre.back(), mom_pre.back(), mls_pre.back(), memb_pre.back(), rf_pre.back(), rm_pre.back(),
                     cen_pre.back()};
    if (b->persistent) {
        int rc = batch_build_persistent(b, bodies, body, lat, order);
        if (rc) return rc;
    }
    b->lat_h = lat;
    b->ref_h = ref;
    b->order_h = order;
    b->steps = 0;
    for (int i = 0; i < nl; ++i) b->base[i] = b->ctx[i]->steps;
    return LBIB_OK;
}

int batch_enqueue(Batch *b, int phase, bool store, cudaStream_t st) {
    cudaError_t e = launch_batch_ib(b->prec, b->T, b->G, phase, st);
    if (e == cudaSuccess && !b->sweep_split) e = launch_batch_sweep(b->prec, b->T, b->G, phase, store ? 1 : 0, st);
    if (e == cudaSuccess && b->sweep_split) {
        // fork the side streams from st, one one-lattice sweep per lattice
        // (largest first, round robin), join back into st
        const int ns = (int)b->side.size(), nl = (int)b->lat_h.size();
        e = cudaEventRecord(b->side_ev[0], st);
        for (int k = 0; k < ns && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->side[k], b->side_ev[0], 0);
        for (int q = 0; q < nl && e == cudaSuccess; ++q) {
            const int i = b->order_h[q];
            const LatRef &r = b->ref_h[(size_t)phase * nl + i];
            e = launch_sweep(b->prec, r.fin, r.fout, r.force, r.stamp, r.d_step, b->lat_h[i], store ? r.fields : nullptr,
                             0, nullptr, r.sr, r.parity, b->nsm, b->side[q % ns]);
        }
        for (int k = 0; k < ns && e == cudaSuccess; ++k) {
            e = cudaEventRecord(b->side_ev[1 + k], b->side[k]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(st, b->side_ev[1 + k], 0);
        }
    }
    if (e != cudaSuccess) return bcuda(b, e, "batch launch");
    return LBIB_OK;
}

int batch_launches_per_step(const Batch *b) {
    int n = 0;
    for (int v : {b->G.mom, b->G.mls, b->G.memb, b->G.rf, b->G.rm, b->G.cen}) n += v > 0;
    return n + (b->sweep_split ? (int)b->lat_h.size() : (b->G.sweep > 0));
}

int batch_capture6(Batch *b) {
    cudaError_t e = cudaStreamBeginCapture(b->s_cap, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return bcuda(b, e, "batch capture");
    int rc = LBIB_OK;
    if (b->persistent) {
        // the queue counters start at zero, then one launch runs the six steps
        e = cudaMemsetAsync(b->pctr, 0, b->pctr_bytes, b->s_cap);
        if (e == cudaSuccess) e = launch_batch_persistent(b->prec, b->T, b->P, b->pgrid, b->s_cap);
        if (e != cudaSuccess) rc = bcuda(b, e, "persistent batch launch");
    }
    for (int k = 0; k < 6 && rc == LBIB_OK && !b->persistent; ++k) rc = batch_enqueue(b, k, false, b->s_cap);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->s_cap, &g);
    if (rc) {
        if (g) cudaGraphDestroy(g);
        return rc;
    }
    if (e != cudaSuccess) return bcuda(b, e, "batch capture end");
    e = cudaGraphInstantiate(&b->g6, g, 0);
    cudaGraphDestroy(g);
    if (e != cudaSuccess) {
        b->g6 = nullptr;
        return bcuda(b, e, "batch graph instantiate");
    }
    return LBIB_OK;
}

// The contexts' host-side state after n batch steps.
void batch_advance_contexts(Batch *b, int n) {
    for (Ctx *c : b->ctx) {
        if (n % 2) std::swap(c->fA, c->fB);
        for (auto &d : c->bodies) {
            d.cur = (d.cur + n) % 3;
            d.bcur ^= (n & 1);
        }
        c->steps += n;
        if (!c->bodies.empty()) c->step_host += (uint32_t)n;
    }
}

Batch *as_batch(void *h) { return static_cast<Batch *>(h); }

}  // namespace

extern "C" {

const char *lbib_batch_last_error(const void *h) {
    if (!h) return g_batch_error.c_str();
    return static_cast<const Batch *>(h)->msg.c_str();
}

int lbib_batch_create(void *const *ctxs, int n, void *stream, void **out) {
    if (!out) return bfail(nullptr, LBIB_EINVAL, "out is NULL");
    *out = nullptr;
    if (!ctxs || n < 1) return bfail(nullptr, LBIB_EINVAL, "a batch needs at least one context");
    Batch *b = new Batch();
    for (int i = 0; i < n; ++i) {
        Ctx *c = static_cast<Ctx *>(ctxs[i]);
        if (!c) {
            delete b;
            return bfail(nullptr, LBIB_EINVAL, "NULL context");
        }
        for (Ctx *o : b->ctx)
            if (o == c) {
                delete b;
                return bfail(nullptr, LBIB_EINVAL, "a context appears twice");
            }
        if (c->err) {
            delete b;
            return bfail(nullptr, c->err, "a context holds an error");
        }
        if (i > 0 && c->prec != b->prec) {
            delete b;
            return bfail(nullptr, LBIB_EINVAL, "the contexts of a batch share one precision");
        }
        b->prec = c->prec;
        b->ctx.push_back(c);
    }
    b->base.assign(n, 0);
    cudaError_t e = cudaSuccess;
    if (stream) {
        b->stream = static_cast<cudaStream_t>(stream);
    } else {
        e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
        b->own_stream = e == cudaSuccess;
    }
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->s_cap, cudaStreamNonBlocking);
    b->side.assign(8, nullptr);
    b->side_ev.assign(9, nullptr);
    for (auto &st : b->side)
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    for (auto &ev : b->side_ev)
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    if (e == cudaSuccess) {
        int dev = 0;
        cudaGetDevice(&dev);
        if (cudaDeviceGetAttribute(&b->nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) b->nsm = 1;
    }
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
    b->ctx_ev.assign(n, nullptr);
    for (int i = 0; i < n && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&b->ctx_ev[i], cudaEventDisableTiming);
    if (e != cudaSuccess) {
        int rc = bcuda(nullptr, e, "batch stream or events");
        lbib_batch_destroy(b);
        return rc;
    }
    for (Ctx *c : b->ctx) sync_ctx(c);  // contexts idle before their tables are taken
    int rc = batch_build(b);
    if (rc) {
        g_batch_error = b->msg;
        lbib_batch_destroy(b);
        return rc;
    }
    *out = b;
    return LBIB_OK;
}

int lbib_batch_step(void *h, int nsteps) {
    Batch *b = as_batch(h);
    if (!b) return LBIB_EINVAL;
    if (nsteps < 0) return bfail(b, LBIB_EINVAL, "nsteps < 0");
    if (nsteps == 0) return LBIB_OK;
    for (size_t i = 0; i < b->ctx.size(); ++i) {
        Ctx *c = b->ctx[i];
        if (c->err) return bfail(b, c->err, "a context of the batch holds an error");
        if (c->steps != b->base[i] + b->steps)
            return bfail(b, LBIB_EINVAL, "a context was stepped outside the batch; rebuild the batch");
        if (!c->bodies.empty() && (uint64_t)c->step_host + (uint64_t)nsteps >= 0xFFFFFFFFull)
            return bfail(b, LBIB_EINVAL, "step counter would wrap; step the context alone once");
        // the batch runs after the work already queued on the context's stream
        cudaEventRecord(b->ctx_ev[i], c->stream);
        cudaStreamWaitEvent(b->stream, b->ctx_ev[i], 0);
    }
    int remaining = nsteps;
    while (remaining > 0) {
        const int phase = (int)(b->steps % 6);
        if (phase == 0 && remaining > 6) {
            if (!b->g6) {
                int rc = batch_capture6(b);
                if (rc) return rc;
            }
            cudaError_t e = cudaGraphLaunch(b->g6, b->stream);
            if (e != cudaSuccess) return bcuda(b, e, "batch graph launch");
            b->steps += 6;
            remaining -= 6;
            b->launches += b->persistent ? 1 : 6 * batch_launches_per_step(b);
        } else {
            int rc = batch_enqueue(b, phase, remaining == 1, b->stream);
            if (rc) return rc;
            b->steps += 1;
            remaining -= 1;
            b->launches += batch_launches_per_step(b);
        }
    }
    batch_advance_contexts(b, nsteps);
    b->total_steps += nsteps;
    for (Ctx *c : b->ctx) {
        // the watchdog of each context whose cadence fell inside these steps,
        // on the state after them
        if (c->watch_every > 0 && c->steps / c->watch_every != (c->steps - nsteps) / c->watch_every) {
            int rc = enqueue_watch(c, b->stream);
            if (rc) return bfail(b, rc, c->msg.c_str());
            b->launches++;
        }
    }
    // later work on each context's stream runs after the batch
    cudaError_t e = cudaEventRecord(b->done, b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "batch event");
    for (Ctx *c : b->ctx) cudaStreamWaitEvent(c->stream, b->done, 0);
    return LBIB_OK;
}

int lbib_batch_sync(void *h) {
    Batch *b = as_batch(h);
    if (!b) return LBIB_EINVAL;
    cudaError_t e = cudaStreamSynchronize(b->stream);
    if (e != cudaSuccess) return bcuda(b, e, "batch sync");
    for (Ctx *c : b->ctx) {
        int rc = sync_ctx(c);
        if (rc) return bfail(b, rc, c->msg.c_str());
    }
    return LBIB_OK;
}

int lbib_batch_counters(void *h, long long *steps, long long *launches) {
    Batch *b = as_batch(h);
    if (!b) return LBIB_EINVAL;
    if (steps) *steps = b->total_steps;
    if (launches) *launches = b->launches;
    return LBIB_OK;
}

int lbib_batch_autotune(void *h, int steps, int *choice) {
    Batch *b = as_batch(h);
    if (!b || steps < 1) return LBIB_EINVAL;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess)
        return bcuda(b, cudaGetLastError(), "autotune events");
    // candidates: the batched sweep in (threads, cells per thread) shapes, or
    // one one-lattice sweep launch per lattice (threads = 0), each with the
    // lattices as given or largest first
    // or the persistent kernel (threads = -1) with sweep tiles of 256 x 4, 8
    // or 16 cells
    const int shapes[][2] = {{128, 1}, {256, 1}, {512, 1}, {128, 4},  {256, 4},
                             {512, 4}, {0, 0},   {-1, 4},  {-1, 8},  {-1, 16}};
    float best = 1e30f;
    int best_t = b->sweep_threads, best_o = b->order, best_c = b->sweep_cpt, best_split = b->sweep_split,
        best_p = b->persistent;
    int rc = LBIB_OK;
    for (int o = 0; o < 2 && !rc; ++o)
        for (const auto &shape : shapes) {
                const int t = shape[0] > 0 ? shape[0] : 256, cp = shape[0] ? shape[1] : 4;
                b->sweep_split = shape[0] == 0;
                b->persistent = shape[0] < 0;
                b->sweep_threads = t;
                b->order = o;
                b->sweep_cpt = cp;
                if ((rc = batch_build(b))) break;
                // untimed: one six-step graph launch (captures the graph), then
                // back to phase 0, so that the timed calls run `steps` graph
                // launches and the field-storing last step, as a long
                // lbib_batch_step does
                if ((rc = lbib_batch_step(h, 12))) break;
                float ms = 1e30f;
                for (int rep = 0; rep < 2 && !rc; ++rep) {
                    cudaEventRecord(e0, b->stream);
                    rc = lbib_batch_step(h, 6 * steps + 1);
                    cudaEventRecord(e1, b->stream);
                    if (!rc) rc = lbib_batch_step(h, 5);  // back to phase 0, untimed
                    cudaEventSynchronize(e1);
                    float t_ms = 0.f;
                    cudaEventElapsedTime(&t_ms, e0, e1);
                    if (t_ms < ms) ms = t_ms;
                }
                if (rc) break;
                if (ms < best) {
                    best = ms;
                    best_t = t;
                    best_o = o;
                    best_c = cp;
                    best_split = b->sweep_split;
                    best_p = b->persistent;
                }
            }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    b->sweep_threads = best_t;
    b->order = best_o;
    b->sweep_cpt = best_c;
    b->sweep_split = best_split;
    b->persistent = best_p;
    int rc2 = batch_build(b);
    if (choice) {
        choice[0] = best_p ? -1 : best_split ? 0 : best_t;
        choice[1] = best_o;
        choice[2] = best_c;
    }
    return rc ? rc : rc2;
}

int lbib_batch_set_persistent(void *h, int enable, double wait_limit_s) {
    Batch *b = as_batch(h);
    if (!b) return LBIB_EINVAL;
    if ((enable != 0 && enable != 1) || !(wait_limit_s >= 0.0) || wait_limit_s > 60.0)
        return bfail(b, LBIB_EINVAL, "persistent: enable 0 or 1, wait limit in [0, 60] s");
    b->persistent = enable;
    b->wait_s = wait_limit_s;
    return batch_build(b);
}

int lbib_batch_set_config(void *h, int threads, int order, int cells_per_thread) {
    Batch *b = as_batch(h);
    if (!b) return LBIB_EINVAL;
    if (threads < 0 || threads > 512 || threads % 32 || order < 0 || order > 1 || cells_per_thread < 1 ||
        cells_per_thread > 16)
        return bfail(b, LBIB_EINVAL, "bad batch configuration");
    b->sweep_split = threads == 0;
    b->sweep_threads = threads ? threads : 256;
    b->order = order;
    b->sweep_cpt = cells_per_thread;
    return batch_build(b);
}

void lbib_batch_destroy(void *h) {
    Batch *b = as_batch(h);
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    batch_free_tables(b);
    for (cudaEvent_t ev : b->ctx_ev)
        if (ev) cudaEventDestroy(ev);
    if (b->done) cudaEventDestroy(b->done);
    if (b->s_cap) cudaStreamDestroy(b->s_cap);
    for (auto st : b->side)
        if (st) cudaStreamDestroy(st);
    for (auto ev : b->side_ev)
        if (ev) cudaEventDestroy(ev);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    delete b;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Checkpoints: the device state of a context (every allocation except the
// scratch and the support moments) and its step counters, restored into a
// context set up the same way (same parameters, same bodies in the same
// order, hence the same allocations).
// ---------------------------------------------------------------------------
namespace {

struct CkpHeader {
    char magic[8];
    int32_t version, prec, nx, ny, nz, nbodies, fa_index, nsaved;
    uint32_t step_host;
    int64_t steps, launches;
};

bool persistent(const Ctx *c, size_t k) {
    return std::find(c->transient.begin(), c->transient.end(), c->allocs[k].first) == c->transient.end();
}

size_t checkpoint_size(const Ctx *c) {
    size_t n = sizeof(CkpHeader) + c->bodies.size() * 4 * sizeof(int32_t);
    for (size_t k = 0; k < c->allocs.size(); ++k)
        if (persistent(c, k)) n += sizeof(uint64_t) + c->allocs[k].second;
    return n;
}

}  // namespace

extern "C" {

int lbib_save(void *h, void *buf, size_t *size) {
    Ctx *c = as_ctx(h);
    if (!c || !size) return LBIB_EINVAL;
    const size_t need = checkpoint_size(c);
    if (!buf) {
        *size = need;
        return LBIB_OK;
    }
    if (*size < need) return fail(c, LBIB_EINVAL, "checkpoint buffer too small (%zu < %zu bytes)", *size, need);
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->s_hi);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->s_lo);
    if (e != cudaSuccess) return cuda_fail(c, e, "checkpoint sync");
    unsigned char *out = static_cast<unsigned char *>(buf);
    CkpHeader hd{};
    std::memcpy(hd.magic, "LBIBCKP1", 8);
    hd.version = 1;
    hd.prec = c->prec;
    hd.nx = c->L.nx;
    hd.ny = c->L.ny;
    hd.nz = c->L.nz;
    hd.nbodies = (int32_t)c->bodies.size();
    hd.fa_index = -1;
    hd.nsaved = 0;
    for (size_t k = 0; k < c->allocs.size(); ++k) {
        if (c->allocs[k].first == c->fA) hd.fa_index = (int32_t)k;
        if (persistent(c, k)) ++hd.nsaved;
    }
    hd.step_host = c->step_host;
    hd.steps = c->steps;
    hd.launches = c->launches;
    std::memcpy(out, &hd, sizeof(hd));
    size_t off = sizeof(hd);
    for (const DevBody &b : c->bodies) {
        const int32_t v[4] = {b.cur, b.bcur, b.nv, b.nt};
        std::memcpy(out + off, v, sizeof(v));
        off += sizeof(v);
    }
    for (size_t k = 0; k < c->allocs.size(); ++k) {
        if (!persistent(c, k)) continue;
        const uint64_t n = c->allocs[k].second;
        std::memcpy(out + off, &n, sizeof(n));
        off += sizeof(n);
        e = cudaMemcpy(out + off, c->allocs[k].first, n, cudaMemcpyDeviceToHost);
        if (e != cudaSuccess) return cuda_fail(c, e, "checkpoint copy");
        off += n;
    }
    *size = off;
    return LBIB_OK;
}

int lbib_load(void *h, const void *buf, size_t size) {
    Ctx *c = as_ctx(h);
    if (!c || !buf) return LBIB_EINVAL;
    const unsigned char *in = static_cast<const unsigned char *>(buf);
    CkpHeader hd{};
    if (size < sizeof(hd)) return fail(c, LBIB_EINVAL, "checkpoint too short");
    std::memcpy(&hd, in, sizeof(hd));
    if (std::memcmp(hd.magic, "LBIBCKP1", 8) != 0 || hd.version != 1)
        return fail(c, LBIB_EINVAL, "not a checkpoint of this library");
    if (hd.prec != c->prec || hd.nx != c->L.nx || hd.ny != c->L.ny || hd.nz != c->L.nz ||
        hd.nbodies != (int32_t)c->bodies.size())
        return fail(c, LBIB_EINVAL, "checkpoint of a differently set-up context (lattice, precision or bodies)");
    size_t off = sizeof(hd);
    std::vector<int32_t> bs(4 * c->bodies.size());
    if (size < off + bs.size() * sizeof(int32_t)) return fail(c, LBIB_EINVAL, "checkpoint too short");
    std::memcpy(bs.data(), in + off, bs.size() * sizeof(int32_t));
    off += bs.size() * sizeof(int32_t);
    for (size_t j = 0; j < c->bodies.size(); ++j)
        if (bs[4 * j + 2] != c->bodies[j].nv || bs[4 * j + 3] != c->bodies[j].nt ||
            bs[4 * j] < 0 || bs[4 * j] > 2 || bs[4 * j + 1] < 0 || bs[4 * j + 1] > 1)
            return fail(c, LBIB_EINVAL, "checkpoint bodies differ from the context's");
    int32_t nsaved = 0;
    for (size_t k = 0; k < c->allocs.size(); ++k) nsaved += persistent(c, k);
    if (nsaved != hd.nsaved || hd.fa_index < 0 || hd.fa_index >= (int32_t)c->allocs.size())
        return fail(c, LBIB_EINVAL, "checkpoint buffers differ from the context's");
    // check every size before copying anything
    size_t o = off;
    for (size_t k = 0; k < c->allocs.size(); ++k) {
        if (!persistent(c, k)) continue;
        uint64_t n = 0;
        if (size < o + sizeof(n)) return fail(c, LBIB_EINVAL, "checkpoint too short");
        std::memcpy(&n, in + o, sizeof(n));
        if (n != c->allocs[k].second || size < o + sizeof(n) + n)
            return fail(c, LBIB_EINVAL, "checkpoint buffers differ from the context's");
        o += sizeof(n) + n;
    }
    cudaError_t e = cudaStreamSynchronize(c->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->s_hi);
    if (e == cudaSuccess) e = cudaStreamSynchronize(c->s_lo);
    if (e != cudaSuccess) return cuda_fail(c, e, "checkpoint sync");
    for (size_t k = 0; k < c->allocs.size(); ++k) {
        if (!persistent(c, k)) continue;
        uint64_t n = 0;
        std::memcpy(&n, in + off, sizeof(n));
        off += sizeof(n);
        e = cudaMemcpy(c->allocs[k].first, in + off, n, cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(c, e, "checkpoint restore");
        off += n;
    }
    invalidate_graphs(c);
    void *fa = c->allocs[hd.fa_index].first;
    if (fa != c->fA) std::swap(c->fA, c->fB);
    for (size_t j = 0; j < c->bodies.size(); ++j) {
        c->bodies[j].cur = bs[4 * j];
        c->bodies[j].bcur = bs[4 * j + 1];
    }
    c->steps = hd.steps;
    c->step_host = hd.step_host;
    c->launches = hd.launches;
    *c->h_err = 0;
    c->err = 0;
    c->msg.clear();
    return check_device_error(c) == LBIB_OK ? LBIB_OK : c->err;
}

}  // extern "C"
