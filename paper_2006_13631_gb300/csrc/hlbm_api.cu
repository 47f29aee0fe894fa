// Host side of the C ABI declared in include/hlbm.h: validation, mesh
// topology (node-triangle incidence, FV rows, wall segments, point-location
// bins), device memory, and the per-step launch sequence.
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "hlbm_dev.cuh"
#include "partition.h"

using namespace hk;

namespace {

hlbm_alloc_fn g_alloc = nullptr;
hlbm_free_fn g_free = nullptr;
void* g_alloc_ctx = nullptr;

constexpr int kWindowMargin = 3;

}  // namespace

struct hlbm {
    int dtype = HLBM_F32;
    cudaStream_t stream = nullptr;
    hlbm_alloc_fn alloc = nullptr;
    hlbm_free_fn release = nullptr;
    void* alloc_ctx = nullptr;
    std::string err;
    std::vector<void*> blocks;

    hlbm_grid_t grid{};
    hlbm_patch_t patch{};
    hlbm_motion_t motion{};
    double tau_s = 0.0;

    // mesh (host copies)
    std::vector<double> xy;
    std::vector<int32_t> tri;
    std::vector<int8_t> kind;
    std::vector<int32_t> row_ptr, col, outer;
    std::vector<int32_t> perm;  // internal node -> caller's node (partition order, see create_impl)
    std::vector<int32_t> part_start;  // the parts of that order (the default FV tiles)
    int n_tiles = 0;
    std::vector<void*> tile_blocks;  // device tables of the current FV tiling
    bool use_smem = false;      // a tile kernel (else the global-memory kernel)
    int fv_kind = HLBM_FV_GLOBAL;  // HLBM_FV_* in use
    int fv_depth = 2;              // deep tiles: sub-steps between exchanges asked for (the largest that fits up to it)
    double mxmin = 0, mxmax = 0, mymin = 0, mymax = 0;
    int nnz = 0, nseg = 0;

    Dev<float> df{};
    Dev<double> dd{};
    // nested lattice levels: lv[k-1] is level k (twice the spacing of level
    // k-1), a window-less lattice with population buffers buf[cur] at its
    // current time and buf[1 - cur] at its next; ref couples it with level k-1
    struct Level {
        Dev<float> df{};
        Dev<double> dd{};
        void* buf[2] = {nullptr, nullptr};
        int cur = 0;
        Refine ref{};
    };
    std::vector<Level> lv;
    void* fbuf[2] = {nullptr, nullptr};  // lattice populations
    void* sbox[2] = {nullptr, nullptr};  // window states
    int8_t* cls[2] = {nullptr, nullptr};
    void* fu[2] = {nullptr, nullptr};    // patch populations
    double* force = nullptr;
    int64_t force_cap = 0;
    unsigned* status = nullptr;
    double* scratch = nullptr;           // 8 doubles for reductions
    // status bits that have reached the host; while any is set, hlbm_step
    // refuses to step (until hlbm_clear_status or hlbm_load)
    unsigned fault = 0;
    unsigned* st_host = nullptr;         // pinned copy queued at the end of each hlbm_step call
    cudaEvent_t st_event = nullptr;      // recorded after that copy
    bool st_pending = false;
    // fault injection for tests (hlbm_inject_fault): the next FV launch runs
    // with this tile never releasing its counter and this spin limit
    int inject_stall_tile = -1;
    long inject_spin_limit = 0;
    // the next step's stream-collide away from the patch, run by the spare
    // warps of the FP32 deep-tile FV kernel (FarArgs): far_ready when the
    // current post-collision buffer's successor already holds it outside
    // far_rect, which the next stream-collide then covers alone
    int overlap = 1;
    // the share of the rows whose far part the FV launch streams: on the
    // 4096^2 workload 0.85 gives 0.669 ms per step, all rows 0.692, 0.7 0.677
    double overlap_share = 0.85;
    unsigned* far_next = nullptr;
    bool far_ready = false;
    int far_rect[4] = {0, 0, 0, 0};
    int far_rows = 0;  // the far part covers rows [0, far_rows) outside far_rect
    // the force of a step runs on a side stream beside the next step's
    // relocation, classification and eq. 178 feed (it reads only the patch
    // after the FV sub-steps); the next FV launch, which rewrites both patch
    // buffers, waits for it, and every hlbm_step call joins it before returning
    cudaStream_t side = nullptr;
    cudaEvent_t ev_fv = nullptr, ev_force = nullptr, ev_move = nullptr, ev_cls = nullptr;
    bool force_pending = false;

    int64_t t = 0;
    double Xprev = 0, Yprev = 0;
    // INDUCED motion: lamina displacement and velocity at t, and the largest
    // velocity the patch's outer nodes allow
    double Yi = 0, Vi = 0, vmax_induced = 0;
    int pbx0 = 0, pby0 = 0;
    int ci = 0;  // cls[ci]: latest class
    int si = 0;  // sbox[si]: state at the current time
    int ui = 0;  // fu[ui]: current patch state
    int fi = 0;  // fbuf[fi]: post-collision populations read next

    // per-phase profiling: event pairs recorded around each phase
    bool profiling = false;
    std::vector<cudaEvent_t> ev_pool;
    std::vector<std::pair<int, int>> ev_marks;  // (phase, index of the start event)
    size_t ev_used = 0;
    double phase_ms[HLBM_N_PHASES] = {0, 0, 0, 0};
    int64_t phase_launches[HLBM_N_PHASES] = {0, 0, 0, 0};
};

namespace {

int fail(hlbm* h, int code, const char* fmt, ...) __attribute__((format(printf, 3, 4)));
int fail(hlbm* h, int code, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    if (h) h->err = buf;
    return code;
}

int cuda_check(hlbm* h, cudaError_t e, const char* what) {
    if (e == cudaSuccess) return HLBM_OK;
    return fail(h, HLBM_ECUDA, "%s: %s", what, cudaGetErrorString(e));
}

void* dev_alloc(hlbm* h, size_t bytes) {
    if (bytes == 0) bytes = 16;
    void* p = nullptr;
    if (h->alloc) {
        p = h->alloc(bytes, (void*)h->stream, h->alloc_ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        p = nullptr;
    }
    if (p) h->blocks.push_back(p);
    return p;
}

void dev_free(hlbm* h, void* p) {
    if (!p) return;
    auto it = std::find(h->blocks.begin(), h->blocks.end(), p);
    if (it != h->blocks.end()) h->blocks.erase(it);
    if (h->release)
        h->release(p, (void*)h->stream, h->alloc_ctx);
    else
        cudaFree(p);
}

template <typename T>
T* upload(hlbm* h, const T* src, size_t count, int* rc) {
    T* p = (T*)dev_alloc(h, count * sizeof(T));
    if (!p) {
        *rc = fail(h, HLBM_ENOMEM, "device allocation of %zu bytes failed", count * sizeof(T));
        return nullptr;
    }
    if (count) {
        cudaError_t e = cudaMemcpyAsync(p, src, count * sizeof(T), cudaMemcpyHostToDevice, h->stream);
        if (e != cudaSuccess) *rc = cuda_check(h, e, "cudaMemcpyAsync");
    }
    return p;
}

// lamina position at integer time t (Sec. 2: y(t) = A sin(w t))
void motion_pos(const hlbm_motion_t& m, int64_t t, double* X, double* Y) {
    double tt = (double)t;
    if (m.kind == HLBM_MOTION_HARMONIC) {
        *X = 0.0;
        *Y = m.A * std::sin(m.omega * tt);
    } else if (m.kind == HLBM_MOTION_UNIFORM) {
        *X = m.vx * tt;
        *Y = m.vy * tt;
    } else {
        *X = 0.0;
        *Y = 0.0;
    }
}

double rect_dist(double x, double y, double a, double b) {
    double qx = std::max(std::fabs(x) - a, 0.0), qy = std::max(std::fabs(y) - b, 0.0);
    return std::sqrt(qx * qx + qy * qy);
}

// window of lattice nodes that follows the patch: covers the mesh bounding
// box at centre (cx, cy) widened by kWindowMargin nodes on every side
// an absorbing layer reaching half way across the lattice it lies on (the
// coarsest level with levels)
bool sponge_too_deep(const hlbm_grid_t* g) {
    const bool lv = g->n_levels > 0 && g->levels;
    const int nx = lv ? g->levels[g->n_levels - 1].nx : g->nx, ny = lv ? g->levels[g->n_levels - 1].ny : g->ny;
    return (g->bc_y == HLBM_BC_OUTFLOW && 2 * g->sponge_rows >= ny) ||
           (g->bc_x == HLBM_BC_OUTFLOW && 2 * g->sponge_rows >= nx);
}

void window_origin(const hlbm* h, double cx, double cy, int* bx0, int* by0) {
    *bx0 = (int)std::floor(cx + h->mxmin) - kWindowMargin;
    *by0 = (int)std::floor(cy + h->mymin) - kWindowMargin;
}

// The lattice nodes a step with its window at (bx0, by0) has to stream
// after its relocation, classification and eq. 178 feed: the window (the
// only nodes those touch) and the nodes pulling from it, with the columns
// widened to multiples of 4 (vector boundaries).  r = {x0, y0, x1, y1}.
void near_rect(int nx, int ny, int bw, int bh, int bx0, int by0, int r[4]) {
    r[0] = std::max(0, ((bx0 - 1) / 4) * 4);
    r[1] = std::max(0, by0 - 1);
    r[2] = std::min(nx, ((bx0 + bw + 1 + 3) / 4) * 4);
    r[3] = std::min(ny, by0 + bh + 1);
}

template <typename T>
Dev<T>& dev_of(hlbm* h);
template <>
Dev<float>& dev_of<float>(hlbm* h) {
    return h->df;
}
template <>
Dev<double>& dev_of<double>(hlbm* h) {
    return h->dd;
}

template <typename T>
Dev<T>& ldev_of(hlbm::Level& L);
template <>
Dev<float>& ldev_of<float>(hlbm::Level& L) {
    return L.df;
}
template <>
Dev<double>& ldev_of<double>(hlbm::Level& L) {
    return L.dd;
}

// Levels around the solver's lattice.  level_step: level k >= 1 streams
// and collides its current buffer into its next.  level_couple: for the
// pair (k, k+1) after a step of the finest lattice that brought the time
// to t1, the restriction of level k onto level k+1 when level k has caught
// up with it (then level k+1's buffers swap), and level k's ring at its new
// time when level k has just stepped.  fine_now is level 0's current buffer.
template <typename T>
void level_step(hlbm* h, int k, cudaStream_t s) {
    hlbm::Level& L = h->lv[k - 1];
    Dev<T>& c = ldev_of<T>(L);
    c.fA = (T*)L.buf[L.cur];
    c.fB = (T*)L.buf[1 - L.cur];
    StepArgs ac{};
    launch_stream_collide<T>(c, ac, s);
    launch_sponge<T>(c, s);  // the coarsest level's absorbing outflow layer, if any
}

template <typename T>
bool level_couple(hlbm* h, int k, int64_t t1, void* fine_now, int bx0, int by0, bool initial, cudaStream_t s) {
    hlbm::Level& C = h->lv[k];  // level k+1
    const bool restrict_now = initial || t1 % ((int64_t)2 << k) == 0;
    const bool ring_now = initial || t1 % ((int64_t)1 << k) == 0;
    if (!ring_now) return false;
    Dev<T>& d = k == 0 ? dev_of<T>(h) : ldev_of<T>(h->lv[k - 1]);
    void* fnow = k == 0 ? fine_now : h->lv[k - 1].buf[h->lv[k - 1].cur];
    Couple cp{};
    if (restrict_now) {
        cp.rsrc = fnow;
        cp.rdst = C.buf[initial ? C.cur : 1 - C.cur];
        cp.bx0 = bx0;
        cp.by0 = by0;
        if (!initial) C.cur = 1 - C.cur;
    }
    const int64_t tk = initial ? 0 : t1 >> k;
    cp.c0 = C.buf[C.cur];
    cp.c1 = (tk & 1) ? C.buf[1 - C.cur] : nullptr;
    cp.ring_dst = fnow;
    launch_couple<T>(d, C.ref, cp, s);
    return true;
}

template <typename T>
void bind(hlbm* h, Dev<T>& d) {
    d.fA = (T*)h->fbuf[h->fi];
    d.fB = (T*)h->fbuf[1 - h->fi];
    d.fu_in = (const T*)h->fu[h->ui];
    d.fu_out = (T*)h->fu[1 - h->ui];
    d.force = h->force;
    d.status = h->status;
}

// start of a profiled phase: returns the index of its start event, or -1
int phase_begin(hlbm* h, cudaStream_t s) {
    if (!h->profiling) return -1;
    while (h->ev_pool.size() < h->ev_used + 2) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return -1;
        h->ev_pool.push_back(e);
    }
    int i = (int)h->ev_used;
    h->ev_used += 2;
    cudaEventRecord(h->ev_pool[i], s);
    return i;
}

void phase_end(hlbm* h, int phase, int i, int launches, cudaStream_t s) {
    if (i < 0) return;
    cudaEventRecord(h->ev_pool[i + 1], s);
    h->ev_marks.push_back({phase, i});
    h->phase_launches[phase] += launches;
}

// fold recorded event pairs into the totals (synchronises the stream)
int phase_collect(hlbm* h) {
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e == cudaSuccess && h->side) e = cudaStreamSynchronize(h->side);
    if (e != cudaSuccess) return cuda_check(h, e, "profile sync");
    for (auto& m : h->ev_marks) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, h->ev_pool[m.second], h->ev_pool[m.second + 1]) == cudaSuccess)
            h->phase_ms[m.first] += ms;
    }
    h->ev_marks.clear();
    h->ev_used = 0;
    return HLBM_OK;
}

// One lattice step is issued in three parts so that a sweep can interleave
// independent solvers: the lattice part (relocation, classification,
// eq. 178 feed, stream-collide, outer-node feed), the FV sub-steps, and the
// force plus the host bookkeeping.  A plain step issues them back to back.
struct PendingStep {
    StepArgs a;
    int ncls;
    double X, Y;
    double Ynext, Vnext;  // INDUCED motion at t+1
};

template <typename T>
int step_lattice(hlbm* h, cudaStream_t s, PendingStep& ps) {
    Dev<T>& d = dev_of<T>(h);
    const int64_t t = h->t;
    // force history capacity
    if (t + 2 > h->force_cap) {
        int64_t cap = std::max<int64_t>(2 * h->force_cap, t + 4096);
        double* nf = (double*)dev_alloc(h, (size_t)cap * 2 * sizeof(double));
        if (!nf) return fail(h, HLBM_ENOMEM, "force history allocation failed");
        cudaMemcpyAsync(nf, h->force, (size_t)h->force_cap * 2 * sizeof(double), cudaMemcpyDeviceToDevice, s);
        cudaStreamSynchronize(s);
        dev_free(h, h->force);
        h->force = nf;
        h->force_cap = cap;
    }
    double X, Y;
    StepArgs a{};
    if (h->motion.kind == HLBM_MOTION_INDUCED) {
        // one symplectic Euler step of the lamina with the force at t
        double f[2];
        cudaError_t e = cudaMemcpyAsync(f, h->force + 2 * t, sizeof f, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) return cuda_check(h, e, "force read-back");
        const hlbm_motion_t& m = h->motion;
        const double acc = (f[1] - m.damping * h->Vi - m.stiffness * h->Yi) / m.mass;
        ps.Vnext = h->Vi + acc;
        ps.Ynext = h->Yi + ps.Vnext;
        if (!std::isfinite(ps.Vnext) || std::fabs(ps.Vnext) > h->vmax_induced)
            return fail(h, HLBM_EINVAL, "step %lld: the lamina's velocity %g exceeds the %g the patch allows",
                        (long long)t, ps.Vnext, h->vmax_induced);
        X = 0.0;
        Y = h->Yi;
        a.v0 = h->Vi;
        a.v1 = ps.Vnext;
    } else {
        motion_pos(h->motion, t, &X, &Y);
    }
    a.t = t;
    a.cx = h->patch.x_c + X;
    a.cy = h->patch.y_c + Y;
    a.dX = X - h->Xprev;
    a.dY = Y - h->Yprev;
    window_origin(h, a.cx, a.cy, &a.bx0, &a.by0);
    a.pbx0 = h->pbx0;
    a.pby0 = h->pby0;
    a.first = (t == 0);
    if (a.bx0 < 1 || a.by0 < 1 || a.bx0 + d.bw > d.nx - 1 || a.by0 + d.bh > d.ny - 1)
        return fail(h, HLBM_EINVAL, "step %lld: the patch window [%d,%d)x[%d,%d) leaves the lattice",
                    (long long)t, a.bx0, a.bx0 + d.bw, a.by0, a.by0 + d.bh);
    if (std::fabs(a.dX) >= 1.0 || std::fabs(a.dY) >= 1.0)
        return fail(h, HLBM_EINVAL, "step %lld: displacement (%g, %g) is not below one lattice spacing",
                    (long long)t, a.dX, a.dY);
    bind(h, d);
    // 1. move the patch to y(t) and refill it (Sec. 4)
    const int ncls = (t == 0) ? h->ci : 1 - h->ci;
    d.cls_prev = h->cls[h->ci];
    d.cls_cur = h->cls[ncls];
    d.sbox_old = (const T*)h->sbox[h->si];
    d.sbox_new = (T*)h->sbox[1 - h->si];
    int ev = phase_begin(h, s);
    if (t > 0) {
        // 2. classify the lattice nodes against the moved fictitious curve: on
        // the side stream beside the refill when the solver steps on its own
        // stream (classification is geometry only, and the class buffer it
        // writes was last read by the previous step's refill and feed)
        const bool cls_side = h->side && s == h->stream;
        if (cls_side) {
            cudaEventRecord(h->ev_move, s);
            cudaStreamWaitEvent(h->side, h->ev_move, 0);
            launch_classify<T>(d, a, h->side);
            cudaEventRecord(h->ev_cls, h->side);
        }
        launch_refill<T>(d, a, s);
        h->ui = 1 - h->ui;
        bind(h, d);
        if (cls_side)
            cudaStreamWaitEvent(s, h->ev_cls, 0);
        else
            launch_classify<T>(d, a, s);
    }
    // 3. interpolation nodes from the patch (eq. postcollision2_s)
    launch_fill<T>(d, a, s);
    phase_end(h, HLBM_PHASE_MOVE, ev, t > 0 ? 3 : 1, s);
    // 4. stream-collide t -> t+1 (eq. LBE)
    ev = phase_begin(h, s);
    int nl = 1;
    // the levels whose step starts now, coarsest first
    for (int k = (int)h->lv.size(); k >= 1; --k)
        if (t % ((int64_t)1 << k) == 0) {
            level_step<T>(h, k, s);
            ++nl;
        }
    int nr[4];
    near_rect(d.nx, d.ny, d.bw, d.bh, a.bx0, a.by0, nr);
    if (h->far_ready && std::equal(nr, nr + 4, h->far_rect)) {
        // the rectangle, and the rows the FV launch left (a node in both is
        // computed twice from the same inputs, to the same values)
        launch_stream_collide_rect<T>(d, a, nr[0], nr[1], nr[2], nr[3], s);
        if (h->far_rows < d.ny) {
            launch_stream_collide_rect<T>(d, a, 0, h->far_rows, d.nx, d.ny, s);
            ++nl;
        }
    } else {
        launch_stream_collide<T>(d, a, s);
    }
    h->far_ready = false;
    nl += launch_sponge<T>(d, s);  // the absorbing outflow layer, if any, on the step's output
    // restrictions (finest first) and the rings of the levels that just stepped
    for (int k = 0; k < (int)h->lv.size(); ++k)
        nl += level_couple<T>(h, k, t + 1, d.fB, a.bx0, a.by0, false, s) ? 1 : 0;
    phase_end(h, HLBM_PHASE_STREAM, ev, nl, s);
    // 5a. the outer nodes' feed from the lattice at t and t+1
    launch_feed<T>(d, a, s);
    ps.a = a;
    ps.ncls = ncls;
    ps.X = X;
    ps.Y = Y;
    return HLBM_OK;
}

// FarArgs of the next step's stream-collide outside its near rectangle, when
// the spare warps of the FV kernel can run it: FP32 lattice, deep-tile FV,
// one lattice level, a prescribed motion (the next window is known)
template <typename T>
bool far_args(hlbm* h, const PendingStep& ps, FarArgs<T>& far) {
    Dev<T>& d = dev_of<T>(h);
    if (!h->overlap || sizeof(T) != 4 || h->dtype != HLBM_F32 || h->fv_kind != HLBM_FV_DEEP || !h->lv.empty() ||
        h->motion.kind == HLBM_MOTION_INDUCED)
        return false;
    double X, Y;
    motion_pos(h->motion, ps.a.t + 1, &X, &Y);
    int bx0, by0;
    window_origin(h, h->patch.x_c + X, h->patch.y_c + Y, &bx0, &by0);
    if (bx0 < 1 || by0 < 1 || bx0 + d.bw > d.nx - 1 || by0 + d.bh > d.ny - 1) return false;
    near_rect(d.nx, d.ny, d.bw, d.bh, bx0, by0, h->far_rect);
    far.src = d.fB;  // the post-collision state at t+1 this step's stream-collide wrote
    far.dst = d.fA;
    far.ex0 = h->far_rect[0];
    far.ey0 = h->far_rect[1];
    far.ex1 = h->far_rect[2];
    far.ey1 = h->far_rect[3];
    far.n_seg = (d.nx + 63) / 64;
    h->far_rows = std::max(1, std::min(d.ny, (int)std::lround(h->overlap_share * d.ny)));
    far.n_chunks = h->far_rows * far.n_seg;
    far.next = h->far_next;
    return true;
}

template <typename T>
int step_fv(hlbm* h, cudaStream_t s, PendingStep& ps, cudaEvent_t ev0 = nullptr, cudaEvent_t ev1 = nullptr,
            bool lookahead = false) {
    Dev<T>& d = dev_of<T>(h);
    // 5b. n FV sub-steps (eq. ulbe, eq. postcollision2_u), with the next
    // step's far stream-collide when lookahead is asked for and possible
    FarArgs<T> far{};
    const bool use_far = lookahead && far_args<T>(h, ps, far);
    if (h->force_pending) {  // the previous step's force still reads a patch buffer
        cudaStreamWaitEvent(s, h->ev_force, 0);
        h->force_pending = false;
    }
    if (use_far) cudaMemsetAsync(h->far_next, 0, sizeof(unsigned), s);
    int ev = phase_begin(h, s);
    if (ev0) cudaEventRecord(ev0, s);
    if (h->inject_stall_tile >= 0) {  // one launch only
        d.stall_tile = h->inject_stall_tile;
        d.spin_limit = h->inject_spin_limit;
        h->inject_stall_tile = -1;
    }
    cudaError_t fe = h->fv_kind == HLBM_FV_DEEP   ? launch_fv_deep<T>(d, ps.a, use_far ? &far : nullptr, s)
                     : h->fv_kind == HLBM_FV_TMEM ? launch_fv_tmem<T>(d, ps.a, s)
                     : h->fv_kind == HLBM_FV_SMEM ? launch_fv_smem<T>(d, ps.a, s)
                                                  : launch_fv_persistent<T>(d, ps.a, s);
    d.stall_tile = -1;
    d.spin_limit = kSpinLimit;
    if (ev1) cudaEventRecord(ev1, s);
    if (fe != cudaSuccess) return cuda_check(h, fe, "FV sub-step launch");
    h->far_ready = use_far;
    // the state after the last sub-step is in the record buffer of the last
    // exchange: fu_out when the number of exchanges is odd
    const int n_exch = h->fv_kind == HLBM_FV_DEEP ? (d.n_sub + d.deep_k - 1) / d.deep_k : d.n_sub;
    if (n_exch & 1) h->ui = 1 - h->ui;
    bind(h, d);
    phase_end(h, HLBM_PHASE_FV, ev, 2, s);
    return HLBM_OK;
}

// the bookkeeping of step_fv when the FV sub-steps ran in a packed launch
template <typename T>
void step_fv_packed_done(hlbm* h) {
    Dev<T>& d = dev_of<T>(h);
    if (d.n_sub & 1) h->ui = 1 - h->ui;
    bind(h, d);
}

template <typename T>
int step_finish(hlbm* h, cudaStream_t s, const PendingStep& ps, bool on_side = false) {
    Dev<T>& d = dev_of<T>(h);
    // 6. force on the lamina at t+1 (on the side stream when asked)
    cudaStream_t fs = s;
    if (on_side && h->side) {
        cudaEventRecord(h->ev_fv, s);
        cudaStreamWaitEvent(h->side, h->ev_fv, 0);
        fs = h->side;
    }
    int ev = phase_begin(h, fs);
    launch_force<T>(d, ps.a.t + 1, fs);
    phase_end(h, HLBM_PHASE_FORCE, ev, d.nseg > 0 ? 2 : 1, fs);
    if (fs != s) {
        cudaEventRecord(h->ev_force, fs);
        h->force_pending = true;
    }
    if (h->ev_used > 4096) {
        int rc = phase_collect(h);
        if (rc != HLBM_OK) return rc;
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(h, e, "kernel launch");
    h->fi = 1 - h->fi;
    h->si = 1 - h->si;
    h->ci = ps.ncls;
    h->pbx0 = ps.a.bx0;
    h->pby0 = ps.a.by0;
    h->Xprev = ps.X;
    h->Yprev = ps.Y;
    if (h->motion.kind == HLBM_MOTION_INDUCED) {
        h->Yi = ps.Ynext;
        h->Vi = ps.Vnext;
    }
    h->t = ps.a.t + 1;
    return HLBM_OK;
}

template <typename T>
int step_impl(hlbm* h, int64_t nsteps) {
    // the force on a side stream, except with INDUCED motion (each step reads
    // the previous force on the host first)
    const bool side = h->motion.kind != HLBM_MOTION_INDUCED;
    if (side && !h->side) {
        if (cudaStreamCreateWithFlags(&h->side, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->ev_fv, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->ev_force, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->ev_move, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->ev_cls, cudaEventDisableTiming) != cudaSuccess)
            return cuda_check(h, cudaGetLastError(), "side stream");
    }
    int rc = HLBM_OK;
    for (int64_t k = 0; k < nsteps && rc == HLBM_OK; ++k) {
        PendingStep ps{};
        rc = step_lattice<T>(h, h->stream, ps);
        if (rc == HLBM_OK) rc = step_fv<T>(h, h->stream, ps, nullptr, nullptr, true);
        if (rc == HLBM_OK) rc = step_finish<T>(h, h->stream, ps, side);
    }
    // join: whatever the caller does next on the solver's stream sees the force
    if (h->force_pending) {
        cudaStreamWaitEvent(h->stream, h->ev_force, 0);
        h->force_pending = false;
    }
    if (rc != HLBM_OK) h->far_ready = false;
    return rc;
}

// Deep-tile tables (k_fv_deep) for the tiles [tile_start[k], tile_start[k+1])
// with K layers of ghost nodes.  Layer 0 is the tile's own nodes; layer j
// the nodes the updates of layer j-1 read (row columns; outer nodes read
// nothing) that are in no earlier layer.  Slots: own nodes whose updates read
// only own nodes (n_a), the other own nodes, then layers 1 .. K, each group
// in the caller's node order (on meshes built layer by layer consecutive
// slots then run along a layer, which spreads a warp's gathers over the
// shared-memory banks).  Sub-step s of a block computes the own nodes and
// layers 1 .. K-1-s.  The tiles a tile waits for are the owners of its
// ghosts and the tiles that hold its nodes as ghosts (symmetric, so that no
// tile can overwrite an exchange buffer a neighbour still reads).  Returns
// false when a tile's computed slots exceed comp_cap.
struct DeepTables {
    int K = 0, slot_cap = 0, ocap = 0;
    std::vector<int32_t> ptr, cnt, gid, optr, rptr, row_gid, lcol, nb_ptr, nb;
    std::vector<int8_t> send;
    std::vector<uint16_t> oslot;
};

bool build_deep_tables(const hlbm* h, const std::vector<int32_t>& tile_start, const std::vector<int32_t>& owner,
                       int K, int comp_cap, DeepTables& D) {
    const int n = h->patch.n_nodes, n_tiles = (int)tile_start.size() - 1;
    D = DeepTables{};
    D.K = K;
    D.ptr.assign(n_tiles + 1, 0);
    D.optr.assign(n_tiles + 1, 0);
    D.rptr.assign(n_tiles + 1, 0);
    D.cnt.assign((size_t)kDeepCnt * n_tiles, 0);
    std::vector<int32_t> loc(n, -1);
    std::vector<int8_t> held(n, 0);  // a node some other tile holds as a ghost
    std::vector<std::vector<int32_t>> nbs(n_tiles);
    auto by_caller = [&](int32_t a, int32_t b) { return h->perm[a] < h->perm[b]; };
    auto reads = [&](int q, auto&& fn) {
        if (h->kind[q] == HLBM_NODE_OUTER) return;
        for (int e = h->row_ptr[q] + 1; e < h->row_ptr[q + 1]; ++e) fn(h->col[e]);
    };
    for (int k = 0; k < n_tiles; ++k) {
        const int p0 = tile_start[k], p1 = tile_start[k + 1];
        std::vector<int32_t> A, B;
        for (int q = p0; q < p1; ++q) {
            bool inside = true;
            reads(q, [&](int c) { inside = inside && c >= p0 && c < p1; });
            (inside ? A : B).push_back(q);
        }
        std::sort(A.begin(), A.end(), by_caller);
        std::sort(B.begin(), B.end(), by_caller);
        std::vector<int32_t> order = A;
        order.insert(order.end(), B.begin(), B.end());
        for (size_t i = 0; i < order.size(); ++i) loc[order[i]] = (int32_t)i;
        std::vector<int> layer_size;
        std::vector<int32_t> prev = order;
        for (int j = 1; j <= K; ++j) {
            std::vector<int32_t> lay;
            for (int32_t q : prev)
                reads(q, [&](int c) {
                    if (loc[c] == -1) {  // not in the tile's slots yet, nor in this layer (-2)
                        loc[c] = -2;
                        lay.push_back(c);
                    }
                });
            std::sort(lay.begin(), lay.end(), by_caller);
            for (int32_t c : lay) {
                loc[c] = (int32_t)order.size();
                order.push_back(c);
                held[c] = 1;
                nbs[k].push_back(owner[c]);
            }
            layer_size.push_back((int)lay.size());
            prev = lay;
        }
        const int n_own = p1 - p0, n_slot = (int)order.size();
        int32_t* c = D.cnt.data() + (size_t)kDeepCnt * k;
        c[0] = (int32_t)A.size();
        c[1] = n_own;
        c[2] = n_slot;
        for (int st = 0; st < K; ++st) {
            int cs = n_own;
            for (int j = 1; j <= K - 1 - st; ++j) cs += layer_size[j - 1];
            c[3 + st] = cs;
        }
        const int n_comp = c[3];
        if (n_comp > comp_cap) return false;
        // computed slots: row images (columns as local slots; outer nodes
        // read none of theirs), outer slots for the staged feed
        for (int x = 0; x < n_comp; ++x) {
            const int q = order[x];
            D.row_gid.push_back(q);
            for (int j = 0; j < kTmemMaxEntries; ++j) {
                const int e = h->row_ptr[q] + 1 + j;
                int lc = x;
                if (e < h->row_ptr[q + 1] && h->kind[q] != HLBM_NODE_OUTER) lc = loc[h->col[e]];
                D.lcol.push_back(lc);
            }
            if (h->kind[q] == HLBM_NODE_OUTER) D.oslot.push_back((uint16_t)x);
        }
        D.gid.insert(D.gid.end(), order.begin(), order.end());
        D.ptr[k + 1] = (int32_t)D.gid.size();
        D.rptr[k + 1] = (int32_t)D.row_gid.size();
        D.optr[k + 1] = (int32_t)D.oslot.size();
        D.slot_cap = std::max(D.slot_cap, n_slot);
        D.ocap = std::max(D.ocap, D.optr[k + 1] - D.optr[k]);
        for (int32_t q : order) loc[q] = -1;
    }
    D.send.assign(D.gid.size(), 0);
    for (int k = 0; k < n_tiles; ++k)
        for (int x = 0; x < tile_start[k + 1] - tile_start[k]; ++x) D.send[D.ptr[k] + x] = held[D.gid[D.ptr[k] + x]];
    // symmetric neighbour sets
    std::vector<std::vector<int32_t>> sym(n_tiles);
    for (int k = 0; k < n_tiles; ++k)
        for (int32_t o : nbs[k]) {
            sym[k].push_back(o);
            sym[o].push_back(k);
        }
    D.nb_ptr.assign(n_tiles + 1, 0);
    for (int k = 0; k < n_tiles; ++k) {
        std::sort(sym[k].begin(), sym[k].end());
        sym[k].erase(std::unique(sym[k].begin(), sym[k].end()), sym[k].end());
        D.nb.insert(D.nb.end(), sym[k].begin(), sym[k].end());
        D.nb_ptr[k + 1] = (int32_t)D.nb.size();
    }
    return true;
}

// FV tiles: equal ranges of the Morton-ordered nodes.  The shared-memory
// kernel runs one block per tile, all co-resident; when a tile and its halo
// do not fit in shared memory the global-memory kernel runs instead, with
// as many tiles as it has co-resident blocks.  Neighbour tiles own a column
// of a tile's rows.  n_tiles_req <= 0 picks one tile per SM (at least 64
// nodes each).  Builds the tile tables, halo lists, ELL matrices with
// tile-local columns, node orders and send flags; previous tables are
// released.  Needs the FV matrices (d.coef).
template <typename T>
int build_tiles(hlbm* h, int n_tiles_req, bool tmem_only = false) {
    Dev<T>& d = dev_of<T>(h);
    cudaStream_t s = h->stream;
    const int n = h->patch.n_nodes;
    int rc = HLBM_OK;
    int sms = 0, devi = 0;
    cudaGetDevice(&devi);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, devi);
    int max_row = 0;
    for (int q = 0; q < n; ++q) max_row = std::max(max_row, h->row_ptr[q + 1] - h->row_ptr[q]);
    std::vector<int32_t> tile_start, owner(n), tile_nb_ptr, tile_nb, halo_ptr, halo_ids;
    int tile_cap = 0, halo_cap = 0;
    auto make_tiles = [&](int nt_) {
        tile_start.assign(nt_ + 1, 0);
        if ((int)h->part_start.size() == nt_ + 1)
            tile_start = h->part_start;  // the parts of the node order
        else
            for (int k = 0; k <= nt_; ++k) tile_start[k] = (int32_t)((int64_t)k * n / nt_);
        for (int k = 0; k < nt_; ++k)
            for (int q = tile_start[k]; q < tile_start[k + 1]; ++q) owner[q] = k;
        tile_nb_ptr.assign(nt_ + 1, 0);
        tile_nb.clear();
        halo_ptr.assign(nt_ + 1, 0);
        halo_ids.clear();
        tile_cap = halo_cap = 0;
        for (int k = 0; k < nt_; ++k) {
            std::vector<int32_t> nb, hl;
            for (int q = tile_start[k]; q < tile_start[k + 1]; ++q)
                for (int e = h->row_ptr[q]; e < h->row_ptr[q + 1]; ++e)
                    if (owner[h->col[e]] != k) {
                        nb.push_back(owner[h->col[e]]);
                        hl.push_back(h->col[e]);
                    }
            std::sort(nb.begin(), nb.end());
            nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
            std::sort(hl.begin(), hl.end());
            hl.erase(std::unique(hl.begin(), hl.end()), hl.end());
            tile_nb.insert(tile_nb.end(), nb.begin(), nb.end());
            tile_nb_ptr[k + 1] = (int32_t)tile_nb.size();
            halo_ids.insert(halo_ids.end(), hl.begin(), hl.end());
            halo_ptr[k + 1] = (int32_t)halo_ids.size();
            tile_cap = std::max(tile_cap, tile_start[k + 1] - tile_start[k]);
            halo_cap = std::max(halo_cap, (int)hl.size());
        }
    };
    int n_tiles = n_tiles_req > 0 ? std::min(n_tiles_req, n) : std::max(1, std::min(sms, (n + 63) / 64));
    make_tiles(n_tiles);
    // outer nodes per tile (their feed is staged in shared memory)
    auto outer_cap = [&]() {
        int cap = 0;
        for (size_t k = 0; k + 1 < tile_start.size(); ++k) {
            int c = 0;
            for (int q = tile_start[k]; q < tile_start[k + 1]; ++q) c += h->kind[q] == HLBM_NODE_OUTER;
            cap = std::max(cap, c);
        }
        return cap;
    };
    const int ocap0 = outer_cap();
    // HLBM_FV_* (0: the fastest that applies); a sweep pack needs the tensor-memory kernel
    const int want = tmem_only ? HLBM_FV_TMEM : h->patch.fv_kernel;
    const bool tiles_ok = tile_cap <= fv_tile_max<T>() && tile_cap + halo_cap < 65536;
    // deep tiles: the deepest exchange interval up to fv_depth that fits
    DeepTables deep;
    bool deep_ok = false;
    if ((want == HLBM_FV_AUTO || want == HLBM_FV_DEEP) && max_row - 1 <= 7 && h->patch.outer_fv == 0) {
        for (int K = std::min(h->fv_depth, kDeepMaxK); K >= 1 && !deep_ok; --K) {
            if (!build_deep_tables(h, tile_start, owner, K, fv_deep_tmem_slots<T>(), deep)) continue;
            deep_ok = deep.slot_cap < 65536 &&
                      fv_deep_tile_capacity<T>(fv_deep_smem_bytes<T>(deep.slot_cap, h->patch.n_sub,
                                                                       std::max(deep.ocap, 1))) >= n_tiles;
        }
    }
    const size_t smem = fv_smem_bytes<T>(tile_cap, std::max(halo_cap, 1), std::max(max_row - 1, 0),
                                         h->patch.n_sub, ocap0);
    const size_t tsmem = fv_tmem_smem_bytes<T>(tile_cap, std::max(halo_cap, 1), h->patch.n_sub, ocap0);
    const bool tmem_ok = !deep_ok && tiles_ok && max_row - 1 <= 7 && h->patch.outer_fv == 0 &&
                         (want == HLBM_FV_AUTO || want == HLBM_FV_TMEM) && fv_tmem_tile_capacity<T>(tsmem) >= n_tiles;
    const bool smem_ok = !deep_ok && !tmem_ok && tiles_ok && (want == HLBM_FV_AUTO || want == HLBM_FV_SMEM) &&
                         fv_smem_tile_capacity<T>(smem) >= n_tiles;
    h->fv_kind = deep_ok ? HLBM_FV_DEEP : tmem_ok ? HLBM_FV_TMEM : smem_ok ? HLBM_FV_SMEM : HLBM_FV_GLOBAL;
    h->use_smem = h->fv_kind != HLBM_FV_GLOBAL;
    if (want != HLBM_FV_AUTO && want != h->fv_kind)
        return fail(h, HLBM_EINVAL, "FV kernel %d cannot run this patch (tiles of %d nodes, rows of %d entries)", want,
                    tile_cap, max_row);
    if (!h->use_smem) {
        int cap = fv_tile_capacity<T>();
        if (cap < 1) return fail(h, HLBM_ECUDA, "the FV kernel cannot be resident on this device");
        n_tiles = std::max(1, std::min(cap, n_tiles_req > 0 ? n_tiles_req : (n + 63) / 64));
        make_tiles(n_tiles);
    }
    // release the previous tables once the stream has finished with them
    cudaStreamSynchronize(s);
    for (void* old : h->tile_blocks) dev_free(h, old);
    h->tile_blocks.clear();
    auto track = [&](void* ptr) {
        if (ptr) h->tile_blocks.push_back(ptr);
        return ptr;
    };
    d.tile_cap = tile_cap;
    d.halo_cap = std::max(halo_cap, 1);
    h->n_tiles = n_tiles;
    d.n_tiles = n_tiles;
    d.tile_start = (int32_t*)track(upload(h, tile_start.data(), tile_start.size(), &rc));
    if (h->fv_kind == HLBM_FV_DEEP) {
        // the deep kernel waits for the symmetric neighbour sets of its K-deep ghost layers
        tile_nb_ptr = deep.nb_ptr;
        tile_nb = deep.nb;
        if (tile_nb.empty()) tile_nb.push_back(0);
        d.deep_k = deep.K;
        d.deep_slot_cap = deep.slot_cap;
        d.deep_ocap = std::max(deep.ocap, 1);
        if (deep.oslot.empty()) deep.oslot.push_back(0);
        d.deep_ptr = (int32_t*)track(upload(h, deep.ptr.data(), deep.ptr.size(), &rc));
        d.deep_cnt = (int32_t*)track(upload(h, deep.cnt.data(), deep.cnt.size(), &rc));
        d.deep_gid = (int32_t*)track(upload(h, deep.gid.data(), deep.gid.size(), &rc));
        d.deep_send = (int8_t*)track(upload(h, deep.send.data(), deep.send.size(), &rc));
        d.deep_optr = (int32_t*)track(upload(h, deep.optr.data(), deep.optr.size(), &rc));
        d.deep_oslot = (uint16_t*)track(upload(h, deep.oslot.data(), deep.oslot.size(), &rc));
        d.deep_rptr = (int32_t*)track(upload(h, deep.rptr.data(), deep.rptr.size(), &rc));
        const int64_t nrow = (int64_t)deep.row_gid.size();
        uint32_t* rows = (uint32_t*)track(dev_alloc(h, std::max<int64_t>(nrow, 1) * fv_deep_row_words<T>() * 4));
        int32_t* d_rgid = upload(h, deep.row_gid.data(), deep.row_gid.size(), &rc);
        int32_t* d_lcol = upload(h, deep.lcol.data(), deep.lcol.size(), &rc);
        if (rc != HLBM_OK) return rc;
        if (!rows || !d_rgid || !d_lcol) return fail(h, HLBM_ENOMEM, "device allocation failed");
        d.deep_rows = rows;
        launch_build_deep_rows<T>(d, d_rgid, d_lcol, nrow, rows, s);
        cudaError_t e3 = cudaStreamSynchronize(s);
        dev_free(h, d_rgid);
        dev_free(h, d_lcol);
        if (e3 != cudaSuccess) return cuda_check(h, e3, "deep tile rows");
    }
    d.tile_nb_ptr = (int32_t*)track(upload(h, tile_nb_ptr.data(), tile_nb_ptr.size(), &rc));
    d.tile_nb = (int32_t*)track(upload(h, tile_nb.data(), tile_nb.size(), &rc));
    // the FV kernel counts sub-steps from t * n_sub (t: the solver's step), so a
    // table rebuilt after some steps starts its counters there
    std::vector<unsigned long long> progress0(n_tiles, (unsigned long long)h->t * (unsigned long long)h->patch.n_sub);
    d.progress = (unsigned long long*)track(upload(h, progress0.data(), progress0.size(), &rc));
    d.halo_ptr = (int32_t*)track(upload(h, halo_ptr.data(), halo_ptr.size(), &rc));
    d.halo_ids = (int32_t*)track(upload(h, halo_ids.data(), halo_ids.size(), &rc));
    // per tile: the processing order of its nodes, those whose rows read only
    // the tile first.  The shared-memory kernel keeps a tile's nodes in this
    // order ("slots"), so the threads of a warp read consecutive slots.
    std::vector<uint16_t> tile_order(std::max(n, 1), 0);  // slot -> tile-local index
    std::vector<int32_t> slot_of(std::max(n, 1), 0);      // node -> slot in its tile
    std::vector<int32_t> tile_interior(n_tiles, 0);
    for (int k = 0; k < n_tiles; ++k) {
        const int p0 = tile_start[k], p1 = tile_start[k + 1];
        std::vector<uint16_t> in, bd;
        for (int q = p0; q < p1; ++q) {
            bool interior = true;
            for (int e = h->row_ptr[q]; e < h->row_ptr[q + 1]; ++e)
                if (h->col[e] < p0 || h->col[e] >= p1) interior = false;
            (interior ? in : bd).push_back((uint16_t)(q - p0));
        }
        // within each group, the caller's node order: meshes built layer by
        // layer (O- and C-grids) then give slots that run along a layer, so
        // the j-th neighbours of consecutive slots are consecutive as well
        // and a warp's gathers spread over the shared-memory banks
        auto by_caller = [&](uint16_t a, uint16_t b) { return h->perm[p0 + a] < h->perm[p0 + b]; };
        std::sort(in.begin(), in.end(), by_caller);
        std::sort(bd.begin(), bd.end(), by_caller);
        tile_interior[k] = (int32_t)in.size();
        std::copy(in.begin(), in.end(), tile_order.begin() + p0);
        std::copy(bd.begin(), bd.end(), tile_order.begin() + p0 + in.size());
        for (int sl = 0; sl < p1 - p0; ++sl) slot_of[p0 + tile_order[p0 + sl]] = sl;
    }
    // ELL layout by slot (columns: slots of the tile, then halo entries) and
    // the nodes other tiles read
    const int ell_w = max_row;
    d.ell_width = ell_w;
    std::vector<int32_t> ell_src((size_t)ell_w * n, -1), ell_col((size_t)ell_w * n, 0);
    std::vector<int8_t> send(n, 0);
    for (int32_t x : halo_ids) send[x] = 1;
    for (int k = 0; k < n_tiles; ++k) {
        const int p0 = tile_start[k], tn = tile_start[k + 1] - p0;
        const int32_t* hb = halo_ids.data() + halo_ptr[k];
        const int hn = halo_ptr[k + 1] - halo_ptr[k];
        for (int sl = 0; sl < tn; ++sl) {
            const int q = p0 + tile_order[p0 + sl];
            for (int j = 0; j < ell_w; ++j) {
                size_t idx = (size_t)ell_w * p0 + (size_t)j * tn + sl;
                int e = h->row_ptr[q] + j;
                if (e < h->row_ptr[q + 1]) {
                    int c = h->col[e];
                    ell_src[idx] = e;
                    if (c >= p0 && c < p0 + tn)
                        ell_col[idx] = slot_of[c];
                    else
                        ell_col[idx] = d.tile_cap + (int)(std::lower_bound(hb, hb + hn, c) - hb);
                } else {
                    ell_col[idx] = sl;
                }
            }
        }
    }
    // per tile: the slots of its outer nodes
    std::vector<int32_t> tile_outer_ptr(n_tiles + 1, 0);
    std::vector<uint16_t> tile_outer_r;
    int ocap = 0;
    for (int k = 0; k < n_tiles; ++k) {
        const int p0 = tile_start[k];
        for (int sl = 0; sl < tile_start[k + 1] - p0; ++sl)
            if (h->kind[p0 + tile_order[p0 + sl]] == HLBM_NODE_OUTER) tile_outer_r.push_back((uint16_t)sl);
        tile_outer_ptr[k + 1] = (int32_t)tile_outer_r.size();
        ocap = std::max(ocap, tile_outer_ptr[k + 1] - tile_outer_ptr[k]);
    }
    if (tile_outer_r.empty()) tile_outer_r.push_back(0);
    d.tile_ocap = ocap;
    d.tile_outer_ptr = (int32_t*)track(upload(h, tile_outer_ptr.data(), tile_outer_ptr.size(), &rc));
    d.tile_outer_r = (uint16_t*)track(upload(h, tile_outer_r.data(), tile_outer_r.size(), &rc));
    d.tile_order = (uint16_t*)track(upload(h, tile_order.data(), tile_order.size(), &rc));
    d.tile_interior = (int32_t*)track(upload(h, tile_interior.data(), tile_interior.size(), &rc));
    d.send = (int8_t*)track(upload(h, send.data(), send.size(), &rc));
    int32_t* d_ell_src = upload(h, ell_src.data(), ell_src.size(), &rc);
    int32_t* d_ell_col = upload(h, ell_col.data(), ell_col.size(), &rc);
    Coef<T>* ellv = (Coef<T>*)track(dev_alloc(h, std::max<size_t>(ell_src.size(), 1) * sizeof(Coef<T>)));
    if (rc != HLBM_OK) return rc;
    if (!ellv || !d.progress || !d_ell_src || !d_ell_col) return fail(h, HLBM_ENOMEM, "device allocation failed");
    d.ell = ellv;
    launch_build_ell<T>(d.coef, d_ell_src, d_ell_col, ellv, (int64_t)ell_src.size(), s);
    cudaError_t e2 = cudaStreamSynchronize(s);
    dev_free(h, d_ell_src);
    dev_free(h, d_ell_col);
    return e2 == cudaSuccess ? HLBM_OK : cuda_check(h, e2, "tile tables");
}

template <typename T>
int create_impl(hlbm* h, const hlbm_grid_t* g) {
    cudaStream_t s = h->stream;
    Dev<T>& d = dev_of<T>(h);
    int rc = HLBM_OK;
    const hlbm_patch_t& p = h->patch;
    const int n = p.n_nodes, nt = p.n_tris;
    d.nx = g->nx;
    d.ny = g->ny;
    d.store = (g->dtype == HLBM_F16 || g->dtype == HLBM_BF16) ? g->dtype : 0;
    d.fscale = g->dtype == HLBM_F16 ? 1024.0f : 1.0f;
    d.finv = 1.0f / d.fscale;
    const size_t lat_elem = g->dtype == HLBM_F16 || g->dtype == HLBM_BF16 ? 2 : sizeof(T);
    d.pitch = (g->nx + 31) / 32 * 32;
    d.plane = (int64_t)d.pitch * g->ny;
    // with levels the boundary kinds belong to the coarsest one; the ring of
    // every finer level is rebuilt every step, whatever its pull wrote
    d.bc_x = g->n_levels ? HLBM_BC_OUTFLOW : g->bc_x;
    d.bc_y = g->n_levels ? HLBM_BC_OUTFLOW : g->bc_y;
    // the absorbing layer belongs to the lattice carrying the domain boundary
    d.sponge_rows = g->n_levels ? 0 : g->sponge_rows;
    d.sponge_sigma = g->n_levels ? 0.0 : g->sponge_sigma;
    d.rho0 = T(g->rho0);
    d.tau_s = T(h->tau_s);
    d.tau_u = T(h->tau_s - 0.5);
    d.inv_tau_u = T(1.0 / (h->tau_s - 0.5));
    d.n_sub = p.n_sub;
    d.outer_fv = p.outer_fv;
    d.dt_u = T(1.0 / p.n_sub);
    d.k178 = T(2.0 * (h->tau_s - 1.0) / (2.0 * h->tau_s - 1.0));
    d.kneq = T(1.0 - 1.0 / (2.0 * h->tau_s));
    d.motion = h->motion.kind;
    d.A = h->motion.A;
    d.omega = h->motion.omega;
    d.vx = h->motion.vx;
    d.vy = h->motion.vy;
    d.half_L = 0.5 * p.lamina_L;
    d.half_T = 0.5 * p.lamina_T;
    d.df2 = p.delta_f * p.delta_f;
    d.n = n;
    d.ntri = nt;

    // --- renumber the nodes so that the default FV tiles (equal parts, one
    // per SM) are compact in graph distance, which sets the size of their
    // halos and ghost layers: recursive bisection of the mesh graph into
    // that many parts, each node set split (in proportion to its parts) by
    // the difference of its BFS distances from two far-apart nodes, so the
    // cut runs across the set's longest extent and follows the mesh around
    // the lamina (nodes on the two faces of the thin lamina are close in
    // space but not in the graph); within a part, Morton order of the
    // positions.  Triangles keep the caller's order (donor ties resolve to
    // the lowest triangle index).
    {
        double hq = 0.0;
        for (int k = 0; k < nt; ++k) {
            const int32_t* v = &h->tri[3 * k];
            hq += 0.5 * std::fabs((h->xy[2 * v[1]] - h->xy[2 * v[0]]) * (h->xy[2 * v[2] + 1] - h->xy[2 * v[0] + 1]) -
                                  (h->xy[2 * v[2]] - h->xy[2 * v[0]]) * (h->xy[2 * v[1] + 1] - h->xy[2 * v[0] + 1]));
        }
        hq = std::sqrt(hq / std::max(n, 1));
        double span = std::max(h->mxmax - h->mxmin, h->mymax - h->mymin);
        if (span / hq > 65000.0) hq = span / 65000.0;
        std::vector<uint64_t> mkey(n);
        for (int i = 0; i < n; ++i) {
            uint32_t ix = (uint32_t)((h->xy[2 * i] - h->mxmin) / hq), iy = (uint32_t)((h->xy[2 * i + 1] - h->mymin) / hq);
            uint64_t k = 0;
            for (int b = 0; b < 16; ++b) k |= (uint64_t)((ix >> b) & 1u) << (2 * b) | (uint64_t)((iy >> b) & 1u) << (2 * b + 1);
            mkey[i] = k;
        }
        int devi = 0, sms = 1;
        cudaGetDevice(&devi);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, devi);
        const int parts = std::max(1, std::min(sms, (n + 63) / 64));
        std::vector<int32_t> order;
        partition_order(n, h->tri.data(), nt, mkey.data(), parts, order, h->part_start);
        h->perm.assign(order.begin(), order.end());
        std::vector<int32_t> inv(n);
        for (int p = 0; p < n; ++p) inv[h->perm[p]] = p;
        std::vector<double> xy2(2 * (size_t)n);
        std::vector<int8_t> kind2(n);
        for (int p = 0; p < n; ++p) {
            xy2[2 * p] = h->xy[2 * h->perm[p]];
            xy2[2 * p + 1] = h->xy[2 * h->perm[p] + 1];
            kind2[p] = h->kind[h->perm[p]];
        }
        for (auto& v : h->tri) v = inv[v];
        h->xy.swap(xy2);
        h->kind.swap(kind2);
    }

    // --- topology: node -> triangles, FV rows (pivot first), wall segments
    std::vector<int32_t> tstart(n + 1, 0), tlist(3 * (size_t)nt);
    for (int k = 0; k < nt; ++k)
        for (int j = 0; j < 3; ++j) tstart[h->tri[3 * k + j] + 1]++;
    for (int i = 0; i < n; ++i) tstart[i + 1] += tstart[i];
    {
        std::vector<int32_t> fill(n, 0);
        for (int k = 0; k < nt; ++k)
            for (int j = 0; j < 3; ++j) {
                int v = h->tri[3 * k + j];
                tlist[tstart[v] + fill[v]++] = k;
            }
    }
    h->row_ptr.assign(n + 1, 0);
    h->col.clear();
    int max_row = 0;
    for (int P = 0; P < n; ++P) {
        std::vector<int32_t> nb;
        for (int e = tstart[P]; e < tstart[P + 1]; ++e)
            for (int j = 0; j < 3; ++j) {
                int v = h->tri[3 * tlist[e] + j];
                if (v != P) nb.push_back(v);
            }
        std::sort(nb.begin(), nb.end());
        nb.erase(std::unique(nb.begin(), nb.end()), nb.end());
        // neighbours counter-clockwise from the +x direction: nodes that are
        // consecutive in the Morton order then read their j-th neighbours in
        // about the same direction, i.e. at nearby, mostly distinct
        // shared-memory banks (exact comparisons, no libm)
        const double px = h->xy[2 * P], py = h->xy[2 * P + 1];
        auto half = [&](int v) {
            const double vx = h->xy[2 * v] - px, vy = h->xy[2 * v + 1] - py;
            return (vy < 0.0 || (vy == 0.0 && vx < 0.0)) ? 1 : 0;
        };
        std::sort(nb.begin(), nb.end(), [&](int a, int b) {
            const int ha = half(a), hb = half(b);
            if (ha != hb) return ha < hb;
            const double ax = h->xy[2 * a] - px, ay = h->xy[2 * a + 1] - py;
            const double bx = h->xy[2 * b] - px, by = h->xy[2 * b + 1] - py;
            const double cr = ax * by - ay * bx;
            if (cr != 0.0) return cr > 0.0;
            return a < b;
        });
        h->col.push_back(P);
        h->col.insert(h->col.end(), nb.begin(), nb.end());
        h->row_ptr[P + 1] = (int32_t)h->col.size();
        max_row = std::max(max_row, (int)nb.size() + 1);
    }
    if (max_row > 64) return fail(h, HLBM_EINVAL, "a patch node has %d neighbours (max 63)", max_row - 1);
    h->nnz = (int)h->col.size();
    d.nnz = h->nnz;
    std::vector<int32_t> outer_of(n, -1);
    h->outer.clear();
    for (int P = 0; P < n; ++P)
        if (h->kind[P] == HLBM_NODE_OUTER) {
            outer_of[P] = (int32_t)h->outer.size();
            h->outer.push_back(P);
        }
    d.n_outer = (int)h->outer.size();
    // wall segments: boundary edges (one incident triangle) joining wall
    // nodes, normal pointing away from the body (towards the third vertex)
    std::vector<int32_t> sa, sb;
    std::vector<double> sn;
    for (int k = 0; k < nt; ++k)
        for (int j = 0; j < 3; ++j) {
            int a = h->tri[3 * k + j], b = h->tri[3 * k + (j + 1) % 3], c = h->tri[3 * k + (j + 2) % 3];
            if (h->kind[a] != HLBM_NODE_WALL || h->kind[b] != HLBM_NODE_WALL) continue;
            int count = 0;
            for (int e = tstart[a]; e < tstart[a + 1]; ++e) {
                const int32_t* v = &h->tri[3 * tlist[e]];
                if (v[0] == b || v[1] == b || v[2] == b) ++count;
            }
            if (count != 1) continue;
            double ex = h->xy[2 * b] - h->xy[2 * a], ey = h->xy[2 * b + 1] - h->xy[2 * a + 1];
            double nx = ey, ny = -ex;
            double tx = h->xy[2 * c] - h->xy[2 * a], ty = h->xy[2 * c + 1] - h->xy[2 * a + 1];
            if (nx * tx + ny * ty < 0) {
                nx = -nx;
                ny = -ny;
            }
            sa.push_back(a);
            sb.push_back(b);
            sn.push_back(nx);
            sn.push_back(ny);
        }
    h->nseg = (int)sa.size();
    d.nseg = h->nseg;

    // --- triangle geometry for barycentric tests, and point-location bins
    std::vector<double> tg(8 * (size_t)nt);
    std::vector<float> tgrad(6 * (size_t)nt);
    double area_sum = 0.0;
    for (int k = 0; k < nt; ++k) {
        const int32_t* v = &h->tri[3 * k];
        double ax = h->xy[2 * v[0]], ay = h->xy[2 * v[0] + 1];
        double x1 = h->xy[2 * v[1]] - ax, y1 = h->xy[2 * v[1] + 1] - ay;
        double x2 = h->xy[2 * v[2]] - ax, y2 = h->xy[2 * v[2] + 1] - ay;
        double det = x1 * y2 - x2 * y1;
        if (!(std::fabs(det) > 0.0)) return fail(h, HLBM_EINVAL, "triangle %d is degenerate", k);
        double* o = &tg[8 * (size_t)k];
        o[0] = ax;
        o[1] = ay;
        o[2] = x1;
        o[3] = y1;
        o[4] = x2;
        o[5] = y2;
        o[6] = det;
        o[7] = 0.0;
        // gradients of the barycentric coordinates (a, b, c) of triangle k
        float* gr = &tgrad[6 * (size_t)k];
        gr[2] = (float)(y2 / det);
        gr[3] = (float)(-x2 / det);
        gr[4] = (float)(-y1 / det);
        gr[5] = (float)(x1 / det);
        gr[0] = (float)(-(y2 - y1) / det);
        gr[1] = (float)((x2 - x1) / det);
        area_sum += 0.5 * std::fabs(det);
    }
    double bh = 1.5 * std::sqrt(area_sum / nt);
    double gx0 = h->mxmin - 1e-6, gy0 = h->mymin - 1e-6;
    int gnx = (int)((h->mxmax + 1e-6 - gx0) / bh) + 1, gny = (int)((h->mymax + 1e-6 - gy0) / bh) + 1;
    std::vector<int32_t> bcount((size_t)gnx * gny + 1, 0), bstart, bitems;
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            bstart.assign((size_t)gnx * gny + 1, 0);
            for (size_t b = 0; b < (size_t)gnx * gny; ++b) bstart[b + 1] = bstart[b] + bcount[b];
            bitems.assign(bstart.back(), 0);
            std::fill(bcount.begin(), bcount.end(), 0);
        }
        for (int k = 0; k < nt; ++k) {
            const int32_t* v = &h->tri[3 * k];
            double lx = 1e300, hx = -1e300, ly = 1e300, hy = -1e300;
            for (int j = 0; j < 3; ++j) {
                lx = std::min(lx, h->xy[2 * v[j]]);
                hx = std::max(hx, h->xy[2 * v[j]]);
                ly = std::min(ly, h->xy[2 * v[j] + 1]);
                hy = std::max(hy, h->xy[2 * v[j] + 1]);
            }
            int i0 = std::max(0, (int)std::floor((lx - 1e-9 - gx0) / bh));
            int i1 = std::min(gnx - 1, (int)std::floor((hx + 1e-9 - gx0) / bh));
            int j0 = std::max(0, (int)std::floor((ly - 1e-9 - gy0) / bh));
            int j1 = std::min(gny - 1, (int)std::floor((hy + 1e-9 - gy0) / bh));
            for (int bj = j0; bj <= j1; ++bj)
                for (int bi = i0; bi <= i1; ++bi) {
                    size_t b = (size_t)bj * gnx + bi;
                    if (pass == 0)
                        bcount[b]++;
                    else
                        bitems[bstart[b] + bcount[b]++] = k;
                }
        }
    }
    d.gbx0 = gx0;
    d.gby0 = gy0;
    d.gbh = bh;
    d.gnbx = gnx;
    d.gnby = gny;

    // --- window size
    d.bw = (int)std::ceil(h->mxmax - h->mxmin) + 2 * kWindowMargin + 2;
    d.bh = (int)std::ceil(h->mymax - h->mymin) + 2 * kWindowMargin + 2;
    d.bplane = (int64_t)d.bw * d.bh;

    // --- device memory
    size_t fbytes = (size_t)9 * d.plane * lat_elem;
    for (int b = 0; b < 2; ++b) {
        h->fbuf[b] = dev_alloc(h, fbytes);
        h->sbox[b] = dev_alloc(h, (size_t)9 * d.bplane * sizeof(T));
        h->cls[b] = (int8_t*)dev_alloc(h, (size_t)d.bplane);
        h->fu[b] = dev_alloc(h, (size_t)kRec * n * sizeof(T));
        if (!h->fbuf[b] || !h->sbox[b] || !h->cls[b] || !h->fu[b])
            return fail(h, HLBM_ENOMEM, "device allocation failed (lattice %zu bytes per buffer)", fbytes);
    }
    h->lv.resize(g->n_levels);
    for (int k = 1; k <= g->n_levels; ++k) {
        const hlbm_level_t& G = g->levels[k - 1];
        hlbm::Level& L = h->lv[k - 1];
        Dev<T>& c = ldev_of<T>(L);
        c = d;
        c.nx = G.nx;
        c.ny = G.ny;
        c.pitch = (G.nx + 31) / 32 * 32;
        c.plane = (int64_t)c.pitch * G.ny;
        const bool coarsest = k == g->n_levels;
        c.bc_x = coarsest ? g->bc_x : HLBM_BC_OUTFLOW;
        c.bc_y = coarsest ? g->bc_y : HLBM_BC_OUTFLOW;
        c.sponge_rows = coarsest ? g->sponge_rows : 0;
        c.sponge_sigma = coarsest ? g->sponge_sigma : 0.0;
        const double tau_f = 0.5 + std::ldexp(h->tau_s - 0.5, -(k - 1)), tau_c = 0.5 + std::ldexp(h->tau_s - 0.5, -k);
        c.tau_s = T(tau_c);
        c.bw = c.bh = 0;  // no window: every node of a coarser level is computed
        c.bplane = 0;
        L.ref.nxc = G.nx;
        L.ref.nyc = G.ny;
        L.ref.pitch = c.pitch;
        L.ref.plane = c.plane;
        L.ref.ox = G.ox;
        L.ref.oy = G.oy;
        L.ref.acf = (tau_f - 1.0) / (2.0 * (tau_c - 1.0));
        L.ref.afc = 2.0 * (tau_c - 1.0) / (tau_f - 1.0);
        const size_t cbytes = (size_t)9 * c.plane * lat_elem;
        for (int b = 0; b < 2; ++b) {
            L.buf[b] = dev_alloc(h, cbytes);
            if (!L.buf[b]) return fail(h, HLBM_ENOMEM, "device allocation failed (level %d, %zu bytes)", k, cbytes);
            cudaMemsetAsync(L.buf[b], 0, cbytes, s);
        }
        L.cur = 0;
    }
    d.xy = upload(h, h->xy.data(), h->xy.size(), &rc);
    d.kind = upload(h, h->kind.data(), h->kind.size(), &rc);
    d.tri = upload(h, h->tri.data(), h->tri.size(), &rc);
    d.trigeo = upload(h, tg.data(), tg.size(), &rc);
    d.trigrad = upload(h, tgrad.data(), tgrad.size(), &rc);
    d.bstart = upload(h, bstart.data(), bstart.size(), &rc);
    d.bitems = upload(h, bitems.data(), bitems.size(), &rc);
    d.row_ptr = upload(h, h->row_ptr.data(), h->row_ptr.size(), &rc);
    d.col = upload(h, h->col.data(), h->col.size(), &rc);
    d.outer = upload(h, h->outer.data(), h->outer.size(), &rc);
    d.outer_of = upload(h, outer_of.data(), outer_of.size(), &rc);
    d.seg_a = upload(h, sa.data(), sa.size(), &rc);
    d.seg_b = upload(h, sb.data(), sb.size(), &rc);
    d.seg_n = upload(h, sn.data(), sn.size(), &rc);
    int32_t* d_tstart = upload(h, tstart.data(), tstart.size(), &rc);
    int32_t* d_tlist = upload(h, tlist.data(), tlist.size(), &rc);
    Coef<T>* coefv = (Coef<T>*)dev_alloc(h, (size_t)h->nnz * sizeof(Coef<T>));
    d.abort_flag = (unsigned*)dev_alloc(h, 16);
    h->far_next = (unsigned*)dev_alloc(h, 16);
    d.snap = (T*)dev_alloc(h, (size_t)24 * std::max(d.n_outer, 1) * sizeof(T));
    d.rtype = (int32_t*)dev_alloc(h, (size_t)n * sizeof(int32_t));
    d.rdonor = (int32_t*)dev_alloc(h, (size_t)n * sizeof(int32_t));
    d.tstart = d_tstart;
    d.tlist = d_tlist;
    d.fcontrib = (double*)dev_alloc(h, (size_t)2 * std::max(h->nseg, 1) * sizeof(double));
    h->status = (unsigned*)dev_alloc(h, 64);
    h->scratch = (double*)dev_alloc(h, 16 * sizeof(double));
    h->force_cap = 4096;
    h->force = (double*)dev_alloc(h, (size_t)h->force_cap * 2 * sizeof(double));
    if (rc != HLBM_OK) return rc;
    if (!coefv || !d.snap || !d.rtype || !d.rdonor || !h->status || !h->scratch || !h->force || !d.fcontrib ||
        !d.abort_flag || !h->far_next)
        return fail(h, HLBM_ENOMEM, "device allocation failed");
    d.coef = coefv;
    d.spin_limit = kSpinLimit;
    d.stall_tile = -1;
    cudaMemsetAsync(d.abort_flag, 0, 16, s);
    cudaMemsetAsync(h->status, 0, 64, s);
    cudaMemsetAsync(d.rtype, 0, (size_t)n * sizeof(int32_t), s);
    cudaMemsetAsync(d.rdonor, 0xff, (size_t)n * sizeof(int32_t), s);
    cudaMemsetAsync(h->force, 0, (size_t)h->force_cap * 2 * sizeof(double), s);
    for (int b = 0; b < 2; ++b) cudaMemsetAsync(h->fbuf[b], 0, fbytes, s);
    h->fi = h->si = h->ui = h->ci = 0;
    bind(h, d);
    launch_fv_coeffs<T>(d, p.lumped, coefv, s);
    rc = build_tiles<T>(h, 0);
    if (rc != HLBM_OK) return rc;

    // --- initial state: equilibrium at the initial density and velocity
    const size_t N = (size_t)g->nx * g->ny;
    double* drho = g->rho_init ? upload(h, g->rho_init, N, &rc) : nullptr;
    double* dux = g->ux_init ? upload(h, g->ux_init, N, &rc) : nullptr;
    double* duy = g->uy_init ? upload(h, g->uy_init, N, &rc) : nullptr;
    if (rc != HLBM_OK) return rc;
    launch_init_struct<T>(d, drho, dux, duy, g->u0x, g->u0y, s);
    double X0, Y0;
    motion_pos(h->motion, 0, &X0, &Y0);
    if (h->motion.kind == HLBM_MOTION_INDUCED) {
        X0 = 0.0;
        Y0 = h->motion.y0;
        h->Yi = h->motion.y0;
        h->Vi = h->motion.v0;
    }
    StepArgs a{};
    a.t = 0;
    a.cx = p.x_c + X0;
    a.cy = p.y_c + Y0;
    window_origin(h, a.cx, a.cy, &a.bx0, &a.by0);
    if (a.bx0 < 1 || a.by0 < 1 || a.bx0 + d.bw > d.nx - 1 || a.by0 + d.bh > d.ny - 1)
        return fail(h, HLBM_EINVAL, "the patch window does not fit in the lattice");
    a.pbx0 = a.bx0;
    a.pby0 = a.by0;
    a.first = 1;
    d.sbox_new = (T*)h->sbox[0];
    launch_init_box<T>(d, a.bx0, a.by0, drho, dux, duy, g->u0x, g->u0y, s);
    d.cls_cur = h->cls[0];
    launch_classify<T>(d, a, s);
    d.sbox_old = (const T*)h->sbox[0];
    launch_patch_init<T>(d, a, s);
    // coarser levels: equilibrium at their initial state, then each takes
    // the initial state of the level inside it (finest first) and rebuilds
    // that level's ring
    std::vector<double*> lvinit;
    for (int k = 1; k <= g->n_levels; ++k) {
        const hlbm_level_t& G = g->levels[k - 1];
        const size_t Nc = (size_t)G.nx * G.ny;
        double* lr = G.rho_init ? upload(h, G.rho_init, Nc, &rc) : nullptr;
        double* lx = G.ux_init ? upload(h, G.ux_init, Nc, &rc) : nullptr;
        double* ly = G.uy_init ? upload(h, G.uy_init, Nc, &rc) : nullptr;
        lvinit.insert(lvinit.end(), {lr, lx, ly});
        if (rc != HLBM_OK) return rc;
        Dev<T>& c = ldev_of<T>(h->lv[k - 1]);
        c.fA = (T*)h->lv[k - 1].buf[0];
        c.fB = (T*)h->lv[k - 1].buf[1];
        launch_init_struct<T>(c, lr, lx, ly, g->u0x, g->u0y, s);
    }
    for (int k = 0; k < g->n_levels; ++k) level_couple<T>(h, k, 0, d.fA, a.bx0, a.by0, true, s);
    // the initial buffers stand for the post-collision state at t = 0: the
    // absorbing layer acts on them as on every later collision
    {
        Dev<T> di = g->n_levels ? ldev_of<T>(h->lv[g->n_levels - 1]) : d;
        di.fB = di.fA;
        launch_sponge<T>(di, s);
    }
    h->ui = 1;  // the type-1 fill wrote the patch into fu[1]
    bind(h, d);
    launch_force<T>(d, 0, s);
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return cuda_check(h, e, "initialisation");
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_check(h, e, "initialisation");
    dev_free(h, drho);
    dev_free(h, dux);
    dev_free(h, duy);
    for (double* p : lvinit) dev_free(h, p);
    h->t = 0;
    h->Xprev = X0;
    h->Yprev = Y0;
    h->pbx0 = a.bx0;
    h->pby0 = a.by0;
    h->ci = 0;
    h->si = 0;
    return HLBM_OK;
}

int sync_status(hlbm* h, unsigned* bits) {
    unsigned v = 0;
    cudaError_t e = cudaMemcpyAsync(&v, h->status, sizeof v, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_check(h, e, "status readback");
    *bits = v;
    h->fault |= v;
    return HLBM_OK;
}

// The error a set of status bits stands for: a neighbour wait that ran out
// (the FV sub-steps of that step were abandoned), a non-finite force (the
// run diverged), or a geometric precondition that failed on the device.
int status_error(hlbm* h, unsigned bits) {
    if (!bits) return HLBM_OK;
    if (bits & HLBM_ST_SYNC_TIMEOUT)
        return fail(h, HLBM_ETIMEOUT, "status 0x%x: an FV tile waited too long for its neighbours; the FV "
                    "sub-steps of that step were abandoned (hlbm_clear_status or hlbm_load to go on)", bits);
    if (bits & HLBM_ST_NONFINITE)
        return fail(h, HLBM_EUNSTABLE, "status 0x%x: the force became NaN/Inf: the run diverged", bits);
    return fail(h, HLBM_EGEOM, "status 0x%x: a geometric precondition failed on the device", bits);
}

// Before hlbm_step queues work: the bits already seen on the host, and the
// copy queued at the end of the previous hlbm_step call if it has arrived
// (never waiting for it).
int check_fault(hlbm* h) {
    if (!h->fault && h->st_pending && cudaEventQuery(h->st_event) == cudaSuccess) {
        h->fault |= *(volatile unsigned*)h->st_host;
        h->st_pending = false;
    }
    cudaGetLastError();  // cudaEventQuery's cudaErrorNotReady is not an error here
    return status_error(h, h->fault);
}

// After hlbm_step queued its work: a copy of the status word that the next
// call can look at without waiting.
void queue_status_copy(hlbm* h) {
    if (!h->st_host) {
        if (cudaHostAlloc((void**)&h->st_host, sizeof(unsigned), cudaHostAllocDefault) != cudaSuccess ||
            cudaEventCreateWithFlags(&h->st_event, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            if (h->st_host) cudaFreeHost(h->st_host);
            h->st_host = nullptr;
            return;
        }
    }
    if (cudaMemcpyAsync(h->st_host, h->status, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream) == cudaSuccess &&
        cudaEventRecord(h->st_event, h->stream) == cudaSuccess)
        h->st_pending = true;
    else
        cudaGetLastError();
}

}  // namespace

namespace {

// ---- checkpoint file: a fixed header, then the dynamic device state -------
// The header records what the state depends on (sizes, physics, a hash of
// the mesh) so that a file is only restored into a solver created from the
// same inputs; everything derived from the inputs at creation (geometry,
// FV matrices, tiles) is rebuilt by hlbm_create, not stored.
struct CkptHeader {
    char magic[8];
    uint32_t version;
    int32_t dtype, nx, ny, n_nodes, n_tris, n_sub, bw, bh, bc_x, bc_y, motion, lumped, outer_fv, pad0;
    double tau_s, rho0, A, omega, vx, vy, lamina_L, lamina_T, x_c, y_c, delta_f;
    uint64_t mesh_hash;
    int64_t t;
    double Xprev, Yprev;
    int32_t pbx0, pby0, ci, si, ui, fi;
    uint32_t status, pad;
    double mass, stiffness, damping, y0, v0;  // INDUCED motion parameters
    int32_t sponge_rows, pad1;
    double sponge_sigma;
    double Yi, Vi;                            // and its state at t
    int32_t n_levels, lv_cur[HLBM_MAX_LEVELS]; // nested levels and their current buffers
    int32_t lv_dim[HLBM_MAX_LEVELS][4];       // nx, ny, ox, oy of each
};
constexpr char kCkptMagic[8] = {'H', 'L', 'B', 'M', 'C', 'K', 'P', 'T'};

uint64_t fnv1a(uint64_t hsh, const void* p, size_t n) {
    const unsigned char* b = (const unsigned char*)p;
    for (size_t i = 0; i < n; ++i) {
        hsh ^= b[i];
        hsh *= 1099511628211ull;
    }
    return hsh;
}

uint64_t mesh_hash(const hlbm* h) {
    uint64_t v = 1469598103934665603ull;
    v = fnv1a(v, h->xy.data(), h->xy.size() * sizeof(double));
    v = fnv1a(v, h->tri.data(), h->tri.size() * sizeof(int32_t));
    v = fnv1a(v, h->kind.data(), h->kind.size());
    return v;
}

template <typename T>
CkptHeader ckpt_header(hlbm* h) {
    Dev<T>& d = dev_of<T>(h);
    CkptHeader c{};
    std::memcpy(c.magic, kCkptMagic, 8);
    c.version = 5;
    c.dtype = h->dtype;
    c.nx = d.nx;
    c.ny = d.ny;
    c.n_nodes = h->patch.n_nodes;
    c.n_tris = h->patch.n_tris;
    c.n_sub = h->patch.n_sub;
    c.bw = d.bw;
    c.bh = d.bh;
    c.bc_x = h->grid.bc_x;
    c.bc_y = h->grid.bc_y;
    c.sponge_rows = h->grid.sponge_rows;
    c.sponge_sigma = h->grid.sponge_sigma;
    c.motion = h->motion.kind;
    c.lumped = h->patch.lumped;
    c.outer_fv = h->patch.outer_fv;
    c.tau_s = h->tau_s;
    c.rho0 = h->grid.rho0;
    c.A = h->motion.A;
    c.omega = h->motion.omega;
    c.vx = h->motion.vx;
    c.vy = h->motion.vy;
    c.lamina_L = h->patch.lamina_L;
    c.lamina_T = h->patch.lamina_T;
    c.x_c = h->patch.x_c;
    c.y_c = h->patch.y_c;
    c.delta_f = h->patch.delta_f;
    c.mesh_hash = mesh_hash(h);
    c.t = h->t;
    c.Xprev = h->Xprev;
    c.Yprev = h->Yprev;
    c.mass = h->motion.mass;
    c.stiffness = h->motion.stiffness;
    c.damping = h->motion.damping;
    c.y0 = h->motion.y0;
    c.v0 = h->motion.v0;
    c.Yi = h->Yi;
    c.Vi = h->Vi;
    c.pbx0 = h->pbx0;
    c.pby0 = h->pby0;
    c.ci = h->ci;
    c.si = h->si;
    c.ui = h->ui;
    c.fi = h->fi;
    c.n_levels = (int32_t)h->lv.size();
    for (size_t k = 0; k < h->lv.size(); ++k) {
        c.lv_cur[k] = h->lv[k].cur;
        c.lv_dim[k][0] = h->lv[k].ref.nxc;
        c.lv_dim[k][1] = h->lv[k].ref.nyc;
        c.lv_dim[k][2] = h->lv[k].ref.ox;
        c.lv_dim[k][3] = h->lv[k].ref.oy;
    }
    return c;
}

// the device buffers of the state, in file order
template <typename T>
std::vector<std::pair<void*, size_t>> ckpt_sections(hlbm* h, int64_t t) {
    Dev<T>& d = dev_of<T>(h);
    const size_t lat = (d.store ? 2 : sizeof(T)) * 9 * (size_t)d.plane;
    const size_t box = sizeof(T) * 9 * (size_t)d.bplane;
    const size_t rec = sizeof(T) * kRec * (size_t)d.n;
    std::vector<std::pair<void*, size_t>> secs = {
        {h->fbuf[0], lat},  {h->fbuf[1], lat},  {h->sbox[0], box},
        {h->sbox[1], box},  {h->cls[0], (size_t)d.bplane}, {h->cls[1], (size_t)d.bplane},
        {h->fu[0], rec},    {h->fu[1], rec},    {d.rtype, sizeof(int32_t) * (size_t)d.n},
        {d.rdonor, sizeof(int32_t) * (size_t)d.n}, {h->force, 2 * sizeof(double) * (size_t)(t + 1)}};
    for (auto& L : h->lv) {
        const size_t clat = (d.store ? 2 : sizeof(T)) * 9 * (size_t)L.ref.plane;
        secs.push_back({L.buf[0], clat});
        secs.push_back({L.buf[1], clat});
    }
    return secs;
}

constexpr size_t kCkptChunk = size_t(64) << 20;

template <typename T>
int save_impl(hlbm* h, const char* path) {
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_check(h, e, "checkpoint sync");
    CkptHeader c = ckpt_header<T>(h);
    unsigned st = 0;
    int rc = sync_status(h, &st);
    if (rc != HLBM_OK) return rc;
    c.status = st;
    FILE* fp = std::fopen(path, "wb");
    if (!fp) return fail(h, HLBM_EIO, "cannot open %s for writing", path);
    bool ok = std::fwrite(&c, sizeof c, 1, fp) == 1;
    std::vector<unsigned char> buf;
    for (auto& sec : ckpt_sections<T>(h, h->t)) {
        for (size_t off = 0; ok && off < sec.second; off += kCkptChunk) {
            const size_t n = std::min(kCkptChunk, sec.second - off);
            buf.resize(n);
            e = cudaMemcpyAsync(buf.data(), (const char*)sec.first + off, n, cudaMemcpyDeviceToHost, h->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
            if (e != cudaSuccess) {
                std::fclose(fp);
                return cuda_check(h, e, "checkpoint read-back");
            }
            ok = std::fwrite(buf.data(), 1, n, fp) == n;
        }
    }
    ok = (std::fclose(fp) == 0) && ok;
    return ok ? HLBM_OK : fail(h, HLBM_EIO, "writing %s failed", path);
}

template <typename T>
int load_impl(hlbm* h, const char* path) {
    FILE* fp = std::fopen(path, "rb");
    if (!fp) return fail(h, HLBM_EIO, "cannot open %s", path);
    CkptHeader c{};
    if (std::fread(&c, sizeof c, 1, fp) != 1 || std::memcmp(c.magic, kCkptMagic, 8) != 0 || c.version != 5) {
        std::fclose(fp);
        return fail(h, HLBM_EIO, "%s is not a solver checkpoint", path);
    }
    const CkptHeader m = ckpt_header<T>(h);
    const bool same = c.dtype == m.dtype && c.nx == m.nx && c.ny == m.ny && c.n_nodes == m.n_nodes &&
                      c.n_tris == m.n_tris && c.n_sub == m.n_sub && c.bw == m.bw && c.bh == m.bh &&
                      c.bc_x == m.bc_x && c.bc_y == m.bc_y && c.motion == m.motion && c.lumped == m.lumped &&
                      c.outer_fv == m.outer_fv && c.mass == m.mass && c.stiffness == m.stiffness &&
                      c.damping == m.damping && c.y0 == m.y0 && c.v0 == m.v0 &&
                      c.sponge_rows == m.sponge_rows && c.sponge_sigma == m.sponge_sigma &&
                      c.tau_s == m.tau_s && c.rho0 == m.rho0 && c.A == m.A && c.omega == m.omega &&
                      c.vx == m.vx && c.vy == m.vy && c.lamina_L == m.lamina_L && c.lamina_T == m.lamina_T &&
                      c.x_c == m.x_c && c.y_c == m.y_c && c.delta_f == m.delta_f && c.mesh_hash == m.mesh_hash &&
                      c.n_levels == m.n_levels && std::memcmp(c.lv_dim, m.lv_dim, sizeof c.lv_dim) == 0;
    int lv_bits = 0;
    for (int k = 0; k < HLBM_MAX_LEVELS; ++k) lv_bits |= c.lv_cur[k];
    if (!same || c.t < 0 || ((c.ci | c.si | c.ui | c.fi | lv_bits) & ~1)) {
        std::fclose(fp);
        return fail(h, HLBM_EINVAL, "%s was written by a solver with other inputs", path);
    }
    // the whole file must be there before anything is overwritten
    size_t want = sizeof c;
    for (auto& sec : ckpt_sections<T>(h, c.t)) want += sec.second;
    long have = -1;
    if (std::fseek(fp, 0, SEEK_END) == 0) have = std::ftell(fp);
    if (have < 0 || (size_t)have != want || std::fseek(fp, (long)sizeof c, SEEK_SET) != 0) {
        std::fclose(fp);
        return fail(h, HLBM_EIO, "%s holds %ld bytes, a checkpoint of this solver at step %lld holds %zu", path,
                    have, (long long)c.t, want);
    }
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) {
        std::fclose(fp);
        return cuda_check(h, e, "checkpoint sync");
    }
    // room for the force history up to t
    if (c.t + 2 > h->force_cap) {
        const int64_t cap = c.t + 4096;
        double* nf = (double*)dev_alloc(h, (size_t)cap * 2 * sizeof(double));
        if (!nf) {
            std::fclose(fp);
            return fail(h, HLBM_ENOMEM, "force history allocation failed");
        }
        cudaMemsetAsync(nf, 0, (size_t)cap * 2 * sizeof(double), h->stream);
        dev_free(h, h->force);
        h->force = nf;
        h->force_cap = cap;
    }
    bool ok = true;
    std::vector<unsigned char> buf;
    for (auto& sec : ckpt_sections<T>(h, c.t)) {
        for (size_t off = 0; ok && off < sec.second; off += kCkptChunk) {
            const size_t n = std::min(kCkptChunk, sec.second - off);
            buf.resize(n);
            ok = std::fread(buf.data(), 1, n, fp) == n;
            if (!ok) break;
            e = cudaMemcpyAsync((char*)sec.first + off, buf.data(), n, cudaMemcpyHostToDevice, h->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
            if (e != cudaSuccess) {
                std::fclose(fp);
                return cuda_check(h, e, "checkpoint upload");
            }
        }
    }
    std::fclose(fp);
    if (!ok) return fail(h, HLBM_EIO, "%s is truncated", path);
    h->t = c.t;
    h->Xprev = c.Xprev;
    h->Yprev = c.Yprev;
    h->Yi = c.Yi;
    h->Vi = c.Vi;
    h->pbx0 = c.pbx0;
    h->pby0 = c.pby0;
    h->ci = c.ci;
    h->si = c.si;
    h->ui = c.ui;
    h->fi = c.fi;
    for (size_t k = 0; k < h->lv.size(); ++k) h->lv[k].cur = c.lv_cur[k];
    Dev<T>& d = dev_of<T>(h);
    e = cudaMemcpyAsync(h->status, &c.status, sizeof(unsigned), cudaMemcpyHostToDevice, h->stream);
    // the FV kernel counts sub-steps from t * n_sub
    std::vector<unsigned long long> prog(d.n_tiles, (unsigned long long)c.t * (unsigned long long)c.n_sub);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(d.progress, prog.data(), prog.size() * sizeof(unsigned long long),
                            cudaMemcpyHostToDevice, h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(d.abort_flag, 0, sizeof(unsigned), h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_check(h, e, "checkpoint state");
    h->fault = c.status;
    h->st_pending = false;
    bind(h, d);
    return HLBM_OK;
}

}  // namespace

namespace {

template <typename T>
int get_fv_impl(hlbm_t* h, const Coef<T>* dcoef, int32_t* row_ptr, int32_t* col, double* gx, double* gy,
                double* cc) {
    const int n = h->patch.n_nodes;
    std::vector<Coef<T>> c(h->nnz);
    cudaError_t e = cudaMemcpyAsync(c.data(), dcoef, c.size() * sizeof(Coef<T>), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_check(h, e, "FV readback");
    std::vector<int32_t> inv(n);
    for (int p = 0; p < n; ++p) inv[h->perm[p]] = p;
    // rows in the caller's numbering: pivot first, then ascending columns
    int pos = 0;
    if (row_ptr) row_ptr[0] = 0;
    for (int P = 0; P < n; ++P) {
        int p = inv[P];
        std::vector<std::pair<int32_t, int>> ent;
        for (int e2 = h->row_ptr[p]; e2 < h->row_ptr[p + 1]; ++e2) {
            int user = h->perm[c[e2].col];
            ent.push_back({user == P ? -1 : user, e2});
        }
        std::sort(ent.begin(), ent.end());
        for (auto& x : ent) {
            if (col) col[pos] = x.first < 0 ? P : x.first;
            if (gx) gx[pos] = double(c[x.second].gx);
            if (gy) gy[pos] = double(c[x.second].gy);
            if (cc) cc[pos] = double(c[x.second].c);
            ++pos;
        }
        if (row_ptr) row_ptr[P + 1] = pos;
    }
    return HLBM_OK;
}

}  // namespace

struct hlbm_sweep {
    std::vector<hlbm*> inst;
    std::vector<cudaStream_t> streams;  // one per instance
    std::vector<cudaEvent_t> ev_lat, ev_fv, ev_done, fv_t0, fv_t1;
    cudaStream_t main = nullptr;        // the caller's stream
    cudaStream_t fv = nullptr;          // FV launches of all instances, one after another
    cudaEvent_t ev_main = nullptr;
    std::vector<double> fv_ms;          // FV time of each instance, summed since the last reset
    std::vector<int32_t> tile_nodes;    // target nodes per FV tile chosen by the tuner (0: default)
    std::vector<std::vector<int>> packs; // instances whose FV sub-steps share one launch
    std::vector<int> pack_of;           // instance -> pack index, -1 when launched alone
    std::vector<cudaEvent_t> ev_pack;   // one per pack: its launch is done
    std::string err;
};

namespace {

int inst_lattice(hlbm* h, cudaStream_t s, PendingStep& ps) {
    return h->dtype != HLBM_F64 ? step_lattice<float>(h, s, ps) : step_lattice<double>(h, s, ps);
}
int inst_fv(hlbm* h, cudaStream_t s, PendingStep& ps, cudaEvent_t e0, cudaEvent_t e1) {
    return h->dtype != HLBM_F64 ? step_fv<float>(h, s, ps, e0, e1) : step_fv<double>(h, s, ps, e0, e1);
}
int inst_finish(hlbm* h, cudaStream_t s, const PendingStep& ps) {
    return h->dtype != HLBM_F64 ? step_finish<float>(h, s, ps) : step_finish<double>(h, s, ps);
}
int inst_retile(hlbm* h, int tiles, bool tmem_only = false) {
    return h->dtype != HLBM_F64 ? build_tiles<float>(h, tiles, tmem_only) : build_tiles<double>(h, tiles, tmem_only);
}

// the tile count of solver i for the tuner's pick (0, the default, before tuning)
int tuned_tiles(const hlbm_sweep* w, int i) {
    const int c = w->tile_nodes[i];
    return c > 0 ? (w->inst[i]->patch.n_nodes + c - 1) / c : 0;
}

// The FV sub-steps of pack p's instances in one cooperative launch of the
// tensor-memory kernel on the sweep's FV stream.
template <typename T>
int pack_fv(hlbm_sweep* w, size_t p, const std::vector<PendingStep>& ps) {
    const std::vector<int>& mem = w->packs[p];
    FvPack<T> pk{};
    pk.n = (int)mem.size();
    int blocks = 0;
    size_t smem = 0;
    for (int k = 0; k < pk.n; ++k) {
        hlbm* h = w->inst[mem[k]];
        Dev<T>& d = dev_of<T>(h);
        pk.block0[k] = blocks;
        pk.d[k] = d;
        pk.a[k] = ps[mem[k]].a;
        pk.g0[k] = (T*)d.fu_in;
        pk.g1[k] = d.fu_out;
        blocks += d.n_tiles;
        smem = std::max(smem, fv_tmem_smem_bytes<T>(d.tile_cap, d.halo_cap, d.n_sub, d.tile_ocap));
    }
    cudaError_t e = launch_fv_tmem_pack<T>(pk, blocks, smem, w->fv);
    if (e != cudaSuccess) {
        w->err = std::string("packed FV launch: ") + cudaGetErrorString(e);
        return HLBM_ECUDA;
    }
    for (int i : mem) step_fv_packed_done<T>(w->inst[i]);
    return HLBM_OK;
}

// One step of every instance.  Instance i issues its lattice part on its
// own stream; the FV sub-steps of all instances run one after another on a
// single stream (each is a cooperative launch that wants the whole GPU, so
// two of them never compete for residency), each as soon as its instance's
// lattice part is done, while other instances' lattice parts run beside
// it; instance i then issues its force on its own stream.
int sweep_one_step(hlbm_sweep* w, bool time_fv) {
    const size_t n = w->inst.size();
    std::vector<PendingStep> ps(n);
    for (size_t i = 0; i < n; ++i) {
        int rc = inst_lattice(w->inst[i], w->streams[i], ps[i]);
        if (rc != HLBM_OK) {
            w->err = "instance " + std::to_string(i) + ": " + w->inst[i]->err;
            return rc;
        }
        cudaEventRecord(w->ev_lat[i], w->streams[i]);
    }
    for (size_t p = 0; p < w->packs.size(); ++p) {
        for (int i : w->packs[p]) cudaStreamWaitEvent(w->fv, w->ev_lat[i], 0);
        int rc = w->inst[w->packs[p][0]]->dtype != HLBM_F64 ? pack_fv<float>(w, p, ps) : pack_fv<double>(w, p, ps);
        if (rc != HLBM_OK) return rc;
        cudaEventRecord(w->ev_pack[p], w->fv);
    }
    for (size_t i = 0; i < n; ++i) {
        if (w->pack_of.size() == n && w->pack_of[i] >= 0) {
            cudaEventRecord(w->ev_fv[i], w->fv);  // after its pack's launch on the same stream
            continue;
        }
        cudaStreamWaitEvent(w->fv, w->ev_lat[i], 0);
        int rc = inst_fv(w->inst[i], w->fv, ps[i], time_fv ? w->fv_t0[i] : nullptr, time_fv ? w->fv_t1[i] : nullptr);
        if (rc != HLBM_OK) {
            w->err = "instance " + std::to_string(i) + ": " + w->inst[i]->err;
            return rc;
        }
        cudaEventRecord(w->ev_fv[i], w->fv);
    }
    for (size_t i = 0; i < n; ++i) {
        cudaStreamWaitEvent(w->streams[i], w->ev_fv[i], 0);
        int rc = inst_finish(w->inst[i], w->streams[i], ps[i]);
        if (rc != HLBM_OK) {
            w->err = "instance " + std::to_string(i) + ": " + w->inst[i]->err;
            return rc;
        }
    }
    if (time_fv) {
        for (size_t i = 0; i < n; ++i) {
            cudaEventSynchronize(w->fv_t1[i]);
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, w->fv_t0[i], w->fv_t1[i]) == cudaSuccess) w->fv_ms[i] += ms;
        }
    }
    return HLBM_OK;
}

}  // namespace

// ---- adjoint of the hybrid step (reverse mode, decisions held fixed) -----
namespace {

// A solver's dynamic state at a step boundary, in device memory.
struct AdjCkpt {
    void* lat = nullptr;  // fbuf[fi]
    void* sbox = nullptr; // sbox[si]
    int8_t* cls = nullptr;
    void* fu = nullptr;   // fu[ui]
    int64_t t = 0;
    double Xprev = 0, Yprev = 0;
    int pbx0 = 0, pby0 = 0, ci = 0, si = 0, ui = 0, fi = 0;
};

// What the reverse of one step needs from its forward pass.
template <typename T>
struct AdjRec {
    StepArgs a{};
    T* P0 = nullptr;   // patch before the refill
    T* Pm = nullptr;   // after it
    T* Pnext = nullptr; // after the FV sub-steps (the patch at t+1)
    T* lat = nullptr;  // lattice populations the stream-collide read (after the eq. 178 fill)
    T* sbo = nullptr;  // window state at t (previous window)
    T* sbn = nullptr;  // at t+1
    int8_t* clp = nullptr;
    int8_t* clc = nullptr;
    int32_t* rt = nullptr;
    int32_t* rd = nullptr;
    T* snap = nullptr;
};

template <typename T>
size_t adj_sizes(hlbm* h, size_t* lat, size_t* box, size_t* fu, size_t* cls) {
    Dev<T>& d = dev_of<T>(h);
    *lat = 9 * (size_t)d.plane * sizeof(T);
    *box = 9 * (size_t)d.bplane * sizeof(T);
    *fu = (size_t)kRec * d.n * sizeof(T);
    *cls = (size_t)d.bplane;
    return *lat;
}

template <typename T>
int adj_snapshot(hlbm* h, AdjCkpt& c, bool restore) {
    size_t lat, box, fu, cls;
    adj_sizes<T>(h, &lat, &box, &fu, &cls);
    cudaStream_t s = h->stream;
    if (restore) {
        h->t = c.t;
        h->Xprev = c.Xprev;
        h->Yprev = c.Yprev;
        h->pbx0 = c.pbx0;
        h->pby0 = c.pby0;
        h->ci = c.ci;
        h->si = c.si;
        h->ui = c.ui;
        h->fi = c.fi;
    }
    auto cp = [&](void* dst, const void* src, size_t n) { return cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToDevice, s); };
    cudaError_t e;
    if (restore) {
        e = cp(h->fbuf[h->fi], c.lat, lat);
        if (e == cudaSuccess) e = cp(h->sbox[h->si], c.sbox, box);
        if (e == cudaSuccess) e = cp(h->cls[h->ci], c.cls, cls);
        if (e == cudaSuccess) e = cp(h->fu[h->ui], c.fu, fu);
        // the FV kernels count sub-steps from t * n_sub
        Dev<T>& d = dev_of<T>(h);
        std::vector<unsigned long long> prog(d.n_tiles, (unsigned long long)h->t * (unsigned long long)d.n_sub);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(d.progress, prog.data(), prog.size() * sizeof(unsigned long long),
                                cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        bind(h, d);
    } else {
        c.t = h->t;
        c.Xprev = h->Xprev;
        c.Yprev = h->Yprev;
        c.pbx0 = h->pbx0;
        c.pby0 = h->pby0;
        c.ci = h->ci;
        c.si = h->si;
        c.ui = h->ui;
        c.fi = h->fi;
        e = cp(c.lat, h->fbuf[h->fi], lat);
        if (e == cudaSuccess) e = cp(c.sbox, h->sbox[h->si], box);
        if (e == cudaSuccess) e = cp(c.cls, h->cls[h->ci], cls);
        if (e == cudaSuccess) e = cp(c.fu, h->fu[h->ui], fu);
    }
    return cuda_check(h, e, "adjoint checkpoint");
}

// one forward step that keeps what its reverse needs
template <typename T>
int adj_forward_step(hlbm* h, AdjRec<T>& R) {
    cudaStream_t s = h->stream;
    Dev<T>& d = dev_of<T>(h);
    size_t lat, box, fu, cls;
    adj_sizes<T>(h, &lat, &box, &fu, &cls);
    auto cp = [&](void* dst, const void* src, size_t n) { cudaMemcpyAsync(dst, src, n, cudaMemcpyDeviceToDevice, s); };
    cp(R.P0, h->fu[h->ui], fu);
    cp(R.sbo, h->sbox[h->si], box);
    cp(R.clp, h->cls[h->ci], cls);
    PendingStep ps{};
    int rc = step_lattice<T>(h, s, ps);
    if (rc != HLBM_OK) return rc;
    R.a = ps.a;
    cp(R.Pm, h->fu[h->ui], fu);
    cp(R.lat, h->fbuf[h->fi], lat);
    cp(R.sbn, h->sbox[1 - h->si], box);
    cp(R.clc, h->cls[ps.ncls], cls);
    cp(R.rt, d.rtype, (size_t)d.n * sizeof(int32_t));
    cp(R.rd, d.rdonor, (size_t)d.n * sizeof(int32_t));
    cp(R.snap, d.snap, (size_t)24 * std::max(d.n_outer, 1) * sizeof(T));
    rc = step_fv<T>(h, s, ps);
    if (rc == HLBM_OK) rc = step_finish<T>(h, s, ps);
    cp(R.Pnext, h->fu[h->ui], fu);
    return rc;
}

// adjoint buffers: adjoints in the population type, parameter sums in FP64
template <typename T>
struct AdjBufs {
    T *lfA, *lfB, *lSo, *lSn, *lPn, *lPm, *lP0, *psi, *x0, *x1, *lsnap;
    double *par, *lY, *lV;
    int32_t* tpos;
};

// reverse of step R.a.t; B.lPn holds the adjoint of the patch at t+1 on entry
// and of the patch at t on exit, B.lfB / lfA and lSn / lSo likewise
template <typename T>
int adj_reverse_step(hlbm* h, const AdjRec<T>& R, AdjBufs<T>& B, T* sub, double lamF) {
    cudaStream_t s = h->stream;
    Dev<T> dd = dev_of<T>(h);
    const int n = dd.n, ns = dd.n_sub;
    const size_t rec = (size_t)kRec * n;
    // the FV sub-steps again (every state kept) and their reverse, one launch;
    // the force at t+1 first, from the state after the last sub-step
    dd.snap = R.snap;
    cudaMemcpyAsync(sub, R.Pm, rec * sizeof(T), cudaMemcpyDeviceToDevice, s);
    cudaMemsetAsync(B.lsnap, 0, (size_t)24 * std::max(dd.n_outer, 1) * sizeof(T), s);
    if (lamF != 0.0) {  // the force at t+1, from the patch after the sub-steps
        dd.fu_in = R.Pnext;
        launch_adj_force<T>(dd, lamF, B.lPn, s);
    }
    cudaError_t fe = launch_adj_fv<T>(dd, R.a, sub, B.lPn, B.x0, B.x1, B.psi, B.tpos, B.lsnap, B.par, B.lV, B.lPm, s);
    if (fe != cudaSuccess) return cuda_check(h, fe, "adjoint FV launch");
    // feed, stream-collide, eq. 178 fill, refill
    dd.sbox_old = R.sbo;
    dd.sbox_new = R.sbn;
    dd.cls_prev = R.clp;
    dd.cls_cur = R.clc;
    cudaMemsetAsync(B.lSo, 0, (size_t)9 * dd.bplane * sizeof(T), s);
    launch_adj_feed<T>(dd, R.a, B.lsnap, B.lSo, B.lSn, B.lY, s);
    cudaMemsetAsync(B.lfA, 0, (size_t)9 * dd.plane * sizeof(T), s);
    dd.fA = R.lat;
    launch_adj_stream<T>(dd, R.a, B.lfB, B.lSn, B.lfA, B.par, s);
    dd.fu_in = R.Pm;
    launch_adj_fill<T>(dd, R.a, B.lfA, B.lPm, B.par, B.lY, s);
    cudaMemsetAsync(B.lP0, 0, (size_t)9 * n * sizeof(T), s);
    if (R.a.t > 0) {
        dd.fu_in = R.P0;
        dd.rtype = R.rt;
        dd.rdonor = R.rd;
        launch_adj_refill<T>(dd, R.a, B.lPm, B.lP0, B.lSo, B.par, B.lY, s);
    }
    std::swap(B.lPn, B.lP0);
    std::swap(B.lfB, B.lfA);
    std::swap(B.lSn, B.lSo);
    cudaError_t e = cudaGetLastError();
    return e == cudaSuccess ? HLBM_OK : cuda_check(h, e, "adjoint launch");
}

// The whole adjoint: forward with checkpoints, Theta, then segments of
// `every` steps recomputed and reversed, last to first.
template <typename T>
int adjoint_impl(hlbm* h, int64_t nsteps, double discard, double fit, double w_re, double w_im, int every,
                 double* theta, double* grad, double* fwd_ms, double* bwd_ms) {
    const double PI = 3.14159265358979323846;
    cudaStream_t s = h->stream;
    Dev<T>& d = dev_of<T>(h);
    const hlbm_motion_t& mo = h->motion;
    const int n = d.n, ns = d.n_sub;
    size_t lat, box, fu, cls;
    adj_sizes<T>(h, &lat, &box, &fu, &cls);
    // transposed row positions: row k's entry of column P -> row P's entry of column k
    std::vector<int32_t> tpos(h->nnz, -1);
    for (int k = 0; k < n; ++k)
        for (int e = h->row_ptr[k] + 1; e < h->row_ptr[k + 1]; ++e) {
            const int P = h->col[e];
            for (int q = h->row_ptr[P] + 1; q < h->row_ptr[P + 1]; ++q)
                if (h->col[q] == k) tpos[e] = q;
            if (tpos[e] < 0) return fail(h, HLBM_EGEOM, "FV rows are not symmetric (node %d, %d)", k, P);
        }
    std::vector<void*> mine;
    auto alloc = [&](size_t bytes) {
        void* p = dev_alloc(h, bytes);
        if (p) mine.push_back(p);
        return p;
    };
    auto release = [&]() {
        cudaStreamSynchronize(s);
        for (void* p : mine) dev_free(h, p);
        mine.clear();
    };
    int rc = HLBM_OK;
    const int64_t nseg = (nsteps + every - 1) / every;
    std::vector<AdjCkpt> ck(nseg);
    for (auto& c : ck) {
        c.lat = alloc(lat);
        c.sbox = alloc(box);
        c.cls = (int8_t*)alloc(cls);
        c.fu = alloc(fu);
        if (!c.lat || !c.sbox || !c.cls || !c.fu) rc = fail(h, HLBM_ENOMEM, "adjoint checkpoints");
    }
    const size_t snapb = (size_t)24 * std::max(d.n_outer, 1) * sizeof(T);
    std::vector<AdjRec<T>> recs(every);
    for (auto& r : recs) {
        r.P0 = (T*)alloc(fu);
        r.Pm = (T*)alloc(fu);
        r.Pnext = (T*)alloc(fu);
        r.lat = (T*)alloc(lat);
        r.sbo = (T*)alloc(box);
        r.sbn = (T*)alloc(box);
        r.clp = (int8_t*)alloc(cls);
        r.clc = (int8_t*)alloc(cls);
        r.rt = (int32_t*)alloc((size_t)n * 4);
        r.rd = (int32_t*)alloc((size_t)n * 4);
        r.snap = (T*)alloc(snapb);
        if (!r.P0 || !r.Pm || !r.Pnext || !r.lat || !r.sbo || !r.sbn || !r.clp || !r.clc || !r.rt || !r.rd || !r.snap)
            rc = fail(h, HLBM_ENOMEM, "adjoint step records");
    }
    AdjBufs<T> B{};
    const size_t z = sizeof(T);
    B.lfA = (T*)alloc(9 * (size_t)d.plane * z);
    B.lfB = (T*)alloc(9 * (size_t)d.plane * z);
    B.lSo = (T*)alloc(9 * (size_t)d.bplane * z);
    B.lSn = (T*)alloc(9 * (size_t)d.bplane * z);
    B.lPn = (T*)alloc(9 * (size_t)n * z);
    B.lPm = (T*)alloc(9 * (size_t)n * z);
    B.lP0 = (T*)alloc(9 * (size_t)n * z);
    B.psi = (T*)alloc(9 * (size_t)n * z);
    B.x0 = (T*)alloc(9 * (size_t)n * z);
    B.x1 = (T*)alloc(9 * (size_t)n * z);
    B.lsnap = (T*)alloc(24 * (size_t)std::max(d.n_outer, 1) * z);
    B.par = (double*)alloc(8 * 8);
    B.lY = (double*)alloc((size_t)(nsteps + 2) * 8);
    B.lV = (double*)alloc((size_t)(nsteps + 1) * ns * 8);
    B.tpos = (int32_t*)alloc((size_t)std::max(h->nnz, 1) * 4);
    T* sub = (T*)alloc((size_t)(ns + 1) * fu);
    if (!B.lfA || !B.lfB || !B.lSo || !B.lSn || !B.lPn || !B.lPm || !B.lP0 || !B.psi || !B.x0 || !B.x1 ||
        !B.lsnap || !B.par || !B.lY || !B.lV || !B.tpos || !sub)
        rc = fail(h, HLBM_ENOMEM, "adjoint buffers");
    if (rc != HLBM_OK) {
        release();
        return rc;
    }
    cudaMemcpyAsync(B.tpos, tpos.data(), tpos.size() * 4, cudaMemcpyHostToDevice, s);
    cudaEvent_t e0, e1, e2;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    cudaEventCreate(&e2);
    // ---- forward, checkpoints every `every` steps
    cudaEventRecord(e0, s);
    for (int64_t t = 0; t < nsteps && rc == HLBM_OK; ++t) {
        if (t % every == 0) rc = adj_snapshot<T>(h, ck[t / every], false);
        if (rc == HLBM_OK) rc = step_impl<T>(h, 1);
    }
    cudaEventRecord(e1, s);
    // ---- Theta and the adjoint of the force history (the fit, Sec. 2.1)
    const double Tp = 2.0 * PI / mo.omega;
    const int64_t t0 = (int64_t)std::ceil(discard * Tp), t1 = (int64_t)std::floor((discard + fit) * Tp);
    if (rc == HLBM_OK && (t1 > nsteps || t1 <= t0 || t0 < 0))
        rc = fail(h, HLBM_EINVAL, "fit window [%lld, %lld] is not inside the %lld steps", (long long)t0,
                  (long long)t1, (long long)nsteps);
    std::vector<double> F(2 * (size_t)(nsteps + 1));
    if (rc == HLBM_OK) {
        cudaError_t e = cudaMemcpyAsync(F.data(), h->force, F.size() * 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_check(h, e, "force history");
    }
    if (rc == HLBM_OK) {
        unsigned st = 0;
        rc = sync_status(h, &st);
        if (rc == HLBM_OK) rc = status_error(h, st);
    }
    std::vector<double> lamF(nsteps + 1, 0.0);
    double gA = 0, gW = 0, gT = 0;
    if (rc == HLBM_OK) {
        const double om = mo.omega, A = mo.A;
        const double N = 0.25 * PI * h->grid.rho0 * om * om * h->patch.lamina_L * h->patch.lamina_L * A;
        double M00 = 0, M01 = 0, M11 = 0, r0 = 0, r1 = 0;
        double dM00 = 0, dM01 = 0, dM11 = 0, dr0 = 0, dr1 = 0;  // d/domega
        for (int64_t t = t0; t <= t1; ++t) {
            const double sn = std::sin(om * t), cs = std::cos(om * t), Fy = F[2 * t + 1], tt = (double)t;
            M00 += sn * sn;
            M01 += sn * cs;
            M11 += cs * cs;
            r0 += Fy * sn;
            r1 += Fy * cs;
            dM00 += 2 * sn * cs * tt;
            dM01 += (cs * cs - sn * sn) * tt;
            dM11 += -2 * sn * cs * tt;
            dr0 += Fy * cs * tt;
            dr1 += -Fy * sn * tt;
        }
        const double det = M00 * M11 - M01 * M01;
        const double a = (r0 * M11 - r1 * M01) / det, b = (r1 * M00 - r0 * M01) / det;
        theta[0] = a / N;
        theta[1] = b / N;
        const double J = w_re * theta[0] + w_im * theta[1];
        // y = M^{-1} v, v = (w_re, w_im) / N
        const double v0 = w_re / N, v1 = w_im / N;
        const double y0 = (v0 * M11 - v1 * M01) / det, y1 = (v1 * M00 - v0 * M01) / det;
        for (int64_t t = t0; t <= t1; ++t) lamF[t] = y0 * std::sin(om * t) + y1 * std::cos(om * t);
        // explicit terms: the basis and N in omega, N in A
        gW = y0 * dr0 + y1 * dr1 - (y0 * (dM00 * a + dM01 * b) + y1 * (dM01 * a + dM11 * b)) - J * 2.0 / om;
        gA = -J / A;
    }
    // ---- reverse sweep by segments
    cudaEventRecord(e2, s);
    if (rc == HLBM_OK) {
        cudaMemsetAsync(B.par, 0, 64, s);
        cudaMemsetAsync(B.lY, 0, (size_t)(nsteps + 2) * 8, s);
        cudaMemsetAsync(B.lV, 0, (size_t)(nsteps + 1) * ns * 8, s);
        cudaMemsetAsync(B.lPn, 0, 9 * (size_t)n * sizeof(T), s);
        cudaMemsetAsync(B.lfB, 0, 9 * (size_t)d.plane * sizeof(T), s);
        cudaMemsetAsync(B.lSn, 0, 9 * (size_t)d.bplane * sizeof(T), s);
    }
    for (int64_t g = nseg - 1; g >= 0 && rc == HLBM_OK; --g) {
        rc = adj_snapshot<T>(h, ck[g], true);
        const int64_t ta = g * every, tb = std::min<int64_t>(nsteps, ta + every);
        for (int64_t t = ta; t < tb && rc == HLBM_OK; ++t) rc = adj_forward_step<T>(h, recs[t - ta]);
        for (int64_t t = tb - 1; t >= ta && rc == HLBM_OK; --t)
            rc = adj_reverse_step<T>(h, recs[t - ta], B, sub, lamF[t + 1]);
    }
    cudaEvent_t e3;
    cudaEventCreate(&e3);
    cudaEventRecord(e3, s);
    if (rc == HLBM_OK) {
        double par[4];
        std::vector<double> lY(nsteps + 2), lV((size_t)(nsteps + 1) * ns);
        cudaError_t e = cudaMemcpyAsync(par, B.par, sizeof par, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(lY.data(), B.lY, lY.size() * 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(lV.data(), B.lV, lV.size() * 8, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        if (e != cudaSuccess) rc = cuda_check(h, e, "adjoint read-back");
        if (rc == HLBM_OK) {
            const double om = mo.omega, A = mo.A, ts = h->tau_s;
            for (int64_t t = 0; t <= nsteps; ++t) {
                gA += lY[t] * std::sin(om * t);
                gW += lY[t] * A * t * std::cos(om * t);
            }
            for (int64_t t = 0; t < nsteps; ++t)
                for (int m = 0; m < ns; ++m) {
                    const double tau = (double)t + double(m + 1) / double(ns), ph = om * tau;
                    const double lv = lV[(size_t)t * ns + m];
                    gA += lv * om * std::cos(ph);
                    gW += lv * (A * std::cos(ph) - A * om * tau * std::sin(ph));
                }
            // tau_s enters as 1/tau_s (BGK), 1/tau_u = 1/(tau_s - 1/2), the eq. 178
            // factor 2 (tau_s - 1)/(2 tau_s - 1) and 1 - 1/(2 tau_s)
            gT = par[0] * (-1.0 / (ts * ts)) + par[1] * (-1.0 / ((ts - 0.5) * (ts - 0.5))) +
                 par[2] * (2.0 / ((2 * ts - 1) * (2 * ts - 1))) + par[3] * (0.5 / (ts * ts));
            grad[0] = gA;
            grad[1] = gW;
            grad[2] = gT;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (fwd_ms) *fwd_ms = ms;
            cudaEventElapsedTime(&ms, e2, e3);
            if (bwd_ms) *bwd_ms = ms;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaEventDestroy(e2);
    cudaEventDestroy(e3);
    release();
    return rc;
}

}  // namespace

extern "C" {

int hlbm_set_allocator(hlbm_alloc_fn alloc, hlbm_free_fn release, void* ctx) {
    if ((alloc == nullptr) != (release == nullptr)) return HLBM_EINVAL;
    g_alloc = alloc;
    g_free = release;
    g_alloc_ctx = ctx;
    return HLBM_OK;
}

namespace {
thread_local std::string g_create_err;
}

int hlbm_create(const hlbm_grid_t* grid, const hlbm_patch_t* patch, double tau_s, const hlbm_motion_t* motion,
                void* cuda_stream, hlbm_t** out) {
    std::string& create_err = g_create_err;
    if (!out) return HLBM_EINVAL;
    *out = nullptr;
    if (!grid || !patch || !motion) return HLBM_EINVAL;
    hlbm* h = new hlbm();
    h->alloc = g_alloc;
    h->release = g_free;
    h->alloc_ctx = g_alloc_ctx;
    h->stream = (cudaStream_t)cuda_stream;
    h->grid = *grid;
    h->patch = *patch;
    h->motion = *motion;
    h->tau_s = tau_s;
    h->dtype = grid->dtype;
    int rc = HLBM_OK;
    const hlbm_patch_t& p = *patch;
    // --- validation (Sec. 3: nu = cs^2 (tau_s - 1/2) = cs^2 tau_u; Sec. 7: dt < 2 tau)
    if (grid->nx < 8 || grid->ny < 8)
        rc = fail(h, HLBM_EINVAL, "lattice %dx%d is too small", grid->nx, grid->ny);
    else if (grid->dtype < HLBM_F64 || grid->dtype > HLBM_BF16)
        rc = fail(h, HLBM_EINVAL, "unknown dtype %d", grid->dtype);
    else if (grid->bc_x < 0 || grid->bc_x > 2 || grid->bc_y < 0 || grid->bc_y > 2)
        rc = fail(h, HLBM_EINVAL, "unknown boundary kind");
    else if (grid->sponge_rows < 0 || !(grid->sponge_sigma >= 0.0 && grid->sponge_sigma < 1.0) ||
             (grid->sponge_rows > 0 && sponge_too_deep(grid)))
        rc = fail(h, HLBM_EINVAL, "absorbing layer of %d rows at strength %g does not fit the lattice",
                  (int)grid->sponge_rows, grid->sponge_sigma);
    else if (!(tau_s > 0.5))
        rc = fail(h, HLBM_EINVAL, "tau_s = %g must exceed 1/2", tau_s);
    else if (p.n_sub < 1 || !(1.0 / p.n_sub < 2.0 * (tau_s - 0.5)))
        rc = fail(h, HLBM_EINVAL, "unstable FV sub-step: dt_u = 1/%d must be below 2 tau_u = %g", p.n_sub,
                  2.0 * (tau_s - 0.5));
    else if (std::fabs(2.0 * tau_s - 1.0) < 1e-12)
        rc = fail(h, HLBM_EINVAL, "tau_s = 1/2 makes eq. 178 singular");
    else if (p.n_nodes < 3 || p.n_tris < 1 || !p.xy || !p.tri || !p.kind)
        rc = fail(h, HLBM_EINVAL, "empty patch mesh");
    else if (motion->kind < 0 || motion->kind > 3)
        rc = fail(h, HLBM_EINVAL, "unknown motion kind %d", motion->kind);
    else if ((p.lumped != 0 && p.lumped != 1) || (p.outer_fv != 0 && p.outer_fv != 1))
        rc = fail(h, HLBM_EINVAL, "lumped = %d and outer_fv = %d must be 0 or 1", p.lumped, p.outer_fv);
    else if (p.fv_kernel < HLBM_FV_AUTO || p.fv_kernel > HLBM_FV_DEEP)
        rc = fail(h, HLBM_EINVAL, "unknown FV kernel %d", p.fv_kernel);
    else if (!(p.delta_f > 1.5))
        rc = fail(h, HLBM_EINVAL, "delta_f = %g must exceed 1.5 (interpolation nodes outside the body)",
                  p.delta_f);
    else if (grid->n_levels < 0 || grid->n_levels > HLBM_MAX_LEVELS || (grid->n_levels && !grid->levels))
        rc = fail(h, HLBM_EINVAL, "n_levels = %d must be 0 .. %d with the levels given", grid->n_levels,
                  HLBM_MAX_LEVELS);
    for (int k = 1; rc == HLBM_OK && k <= grid->n_levels; ++k) {
        // level k-1 (the box) inside level k
        const hlbm_level_t& G = grid->levels[k - 1];
        const int bx = k == 1 ? grid->nx : grid->levels[k - 2].nx, by = k == 1 ? grid->ny : grid->levels[k - 2].ny;
        const int m = k == grid->n_levels ? 1 : 2;
        if (bx % 2 == 0 || by % 2 == 0 || bx < 9 || by < 9 || G.ox < m || G.oy < m ||
            G.ox + (bx + 1) / 2 > G.nx - m || G.oy + (by + 1) / 2 > G.ny - m)
            rc = fail(h, HLBM_EINVAL,
                      "level %d: the %dx%d box at node (%d, %d) must have odd sizes >= 9 and keep %d node(s) to the "
                      "edges of the %dx%d level around it",
                      k - 1, bx, by, G.ox, G.oy, m, G.nx, G.ny);
    }
    for (int k = 0; rc == HLBM_OK && grid->n_levels > 0 && k <= grid->n_levels; ++k) {
        const double tk = 0.5 + std::ldexp(tau_s - 0.5, -k);
        if (std::fabs(tk - 1.0) <= 1e-3)
            rc = fail(h, HLBM_EINVAL, "tau of level %d is %g: the f^neq rescaling between levels needs tau != 1", k,
                      tk);
    }
    if (rc == HLBM_OK) {
        h->xy.assign(p.xy, p.xy + 2 * (size_t)p.n_nodes);
        h->tri.assign(p.tri, p.tri + 3 * (size_t)p.n_tris);
        h->kind.assign(p.kind, p.kind + p.n_nodes);
        for (size_t k = 0; k < h->tri.size() && rc == HLBM_OK; ++k)
            if (h->tri[k] < 0 || h->tri[k] >= p.n_nodes) rc = fail(h, HLBM_EINVAL, "triangle index out of range");
        for (int i = 0; i < p.n_nodes && rc == HLBM_OK; ++i)
            if (h->kind[i] < 0 || h->kind[i] > 2) rc = fail(h, HLBM_EINVAL, "node %d has kind %d", i, h->kind[i]);
    }
    if (rc == HLBM_OK) {
        h->mxmin = h->mymin = 1e300;
        h->mxmax = h->mymax = -1e300;
        double dmin_outer = 1e300;
        for (int i = 0; i < p.n_nodes; ++i) {
            double x = h->xy[2 * i], y = h->xy[2 * i + 1];
            h->mxmin = std::min(h->mxmin, x);
            h->mxmax = std::max(h->mxmax, x);
            h->mymin = std::min(h->mymin, y);
            h->mymax = std::max(h->mymax, y);
            if (h->kind[i] == HLBM_NODE_OUTER)
                dmin_outer = std::min(dmin_outer, rect_dist(x, y, 0.5 * p.lamina_L, 0.5 * p.lamina_T));
        }
        double dmax = 0.0;
        if (motion->kind == HLBM_MOTION_HARMONIC) dmax = std::fabs(motion->A * motion->omega);
        if (motion->kind == HLBM_MOTION_UNIFORM) dmax = std::hypot(motion->vx, motion->vy);
        if (motion->kind == HLBM_MOTION_INDUCED) {
            dmax = std::fabs(motion->v0);
            h->vmax_induced = std::min(0.999, dmin_outer - p.delta_f - 1.5);
            if (!(motion->mass > 0.0) || !std::isfinite(motion->mass) || !(motion->stiffness >= 0.0) ||
                !(motion->damping >= 0.0) || !std::isfinite(motion->stiffness) || !std::isfinite(motion->damping) ||
                !std::isfinite(motion->y0) || !std::isfinite(motion->v0))
                rc = fail(h, HLBM_EINVAL, "INDUCED motion needs mass > 0, stiffness >= 0, damping >= 0, finite y0, v0");
        }
        // outer nodes' bilinear donors (within sqrt 2 < 1.5 of the node) must
        // be discretization nodes at t and t+1
        if (dmin_outer < 1e299 && !(dmin_outer > p.delta_f + 1.5 + dmax))
            rc = fail(h, HLBM_EINVAL,
                      "outer patch boundary at distance %g from the lamina; needs > delta_f + 1.5 + %g", dmin_outer,
                      dmax);
        if (dmax >= 1.0) rc = fail(h, HLBM_EINVAL, "lamina moves %g >= 1 lattice spacing per step", dmax);
        if (motion->kind == HLBM_MOTION_HARMONIC) {
            int bw = (int)std::ceil(h->mxmax - h->mxmin) + 2 * kWindowMargin + 2;
            int bh = (int)std::ceil(h->mymax - h->mymin) + 2 * kWindowMargin + 2;
            for (int sgn = -1; sgn <= 1 && rc == HLBM_OK; sgn += 2) {
                int bx0, by0;
                window_origin(h, p.x_c, p.y_c + sgn * std::fabs(motion->A), &bx0, &by0);
                if (bx0 < 1 || by0 < 1 || bx0 + bw > grid->nx - 1 || by0 + bh > grid->ny - 1)
                    rc = fail(h, HLBM_EINVAL, "the oscillating patch comes within %d nodes of the lattice edge",
                              kWindowMargin);
            }
        }
    }
    if (rc == HLBM_OK) rc = (grid->dtype == HLBM_F64) ? create_impl<double>(h, grid) : create_impl<float>(h, grid);
    if (rc != HLBM_OK) {
        create_err = h->err;
        cudaStreamSynchronize(h->stream);
        for (void* b : std::vector<void*>(h->blocks)) dev_free(h, b);
        delete h;
        return rc;
    }
    *out = h;
    return HLBM_OK;
}

int hlbm_step(hlbm_t* h, int64_t nsteps) {
    if (!h || nsteps < 0) return HLBM_EINVAL;
    int rc = check_fault(h);
    if (rc != HLBM_OK) return rc;
    rc = h->dtype != HLBM_F64 ? step_impl<float>(h, nsteps) : step_impl<double>(h, nsteps);
    if (nsteps > 0) queue_status_copy(h);
    return rc;
}

int hlbm_set_fv_depth(hlbm_t* h, int32_t depth) {
    if (!h) return HLBM_EINVAL;
    if (depth < 1 || depth > HLBM_FV_MAX_DEPTH || depth > kDeepMaxK)
        return fail(h, HLBM_EINVAL, "FV exchange interval %d is not in 1 .. %d", (int)depth, HLBM_FV_MAX_DEPTH);
    h->fv_depth = depth;
    return h->dtype != HLBM_F64 ? build_tiles<float>(h, 0) : build_tiles<double>(h, 0);
}

int hlbm_clear_status(hlbm_t* h) {
    if (!h) return HLBM_EINVAL;
    cudaError_t e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_check(h, e, "clear status");
    const int n_tiles = h->dtype != HLBM_F64 ? h->df.n_tiles : h->dd.n_tiles;
    unsigned long long* prog = h->dtype != HLBM_F64 ? h->df.progress : h->dd.progress;
    unsigned* abort_flag = h->dtype != HLBM_F64 ? h->df.abort_flag : h->dd.abort_flag;
    // the FV kernels count sub-steps from t * n_sub (an abandoned step left
    // the counters anywhere in its range)
    std::vector<unsigned long long> p0(n_tiles, (unsigned long long)h->t * (unsigned long long)h->patch.n_sub);
    e = cudaMemsetAsync(h->status, 0, sizeof(unsigned), h->stream);
    if (e == cudaSuccess) e = cudaMemsetAsync(abort_flag, 0, sizeof(unsigned), h->stream);
    if (e == cudaSuccess && n_tiles)
        e = cudaMemcpyAsync(prog, p0.data(), p0.size() * sizeof(unsigned long long), cudaMemcpyHostToDevice,
                            h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_check(h, e, "clear status");
    h->fault = 0;
    h->st_pending = false;
    h->far_ready = false;  // the next stream-collide covers the whole lattice
    return HLBM_OK;
}

int hlbm_set_overlap(hlbm_t* h, int32_t enable) {
    if (!h) return HLBM_EINVAL;
    h->overlap = enable ? 1 : 0;
    return HLBM_OK;
}

int hlbm_set_overlap_share(hlbm_t* h, double share) {
    if (!h) return HLBM_EINVAL;
    if (!(share > 0.0 && share <= 1.0)) return fail(h, HLBM_EINVAL, "overlap share %g is not in (0, 1]", share);
    h->overlap_share = share;
    return HLBM_OK;
}

int hlbm_inject_fault(hlbm_t* h, int32_t kind, int64_t arg) {
    if (!h) return HLBM_EINVAL;
    if (kind == HLBM_FAULT_STALL_TILE) {
        const int n_tiles = h->dtype != HLBM_F64 ? h->df.n_tiles : h->dd.n_tiles;
        if (arg < 0 || arg >= n_tiles) return fail(h, HLBM_EINVAL, "no FV tile %lld", (long long)arg);
        h->inject_stall_tile = (int)arg;
        h->inject_spin_limit = 1L << 12;
        return HLBM_OK;
    }
    if (kind == HLBM_FAULT_NAN_LATTICE) {
        h->far_ready = false;  // the next stream-collide must read the planted value everywhere
        const int nx = h->grid.nx, ny = h->grid.ny;
        if (arg < 0 || arg >= (int64_t)nx * ny) return fail(h, HLBM_EINVAL, "no lattice node %lld", (long long)arg);
        const int64_t pitch = h->dtype != HLBM_F64 ? h->df.pitch : h->dd.pitch;
        const int64_t plane = h->dtype != HLBM_F64 ? h->df.plane : h->dd.plane;
        const int64_t x = arg % nx, y = arg / nx;
        // a quiet NaN in the storage type of the populations read next
        size_t es;
        unsigned char nan[8];
        if (h->dtype == HLBM_F64) {
            const uint64_t v = 0x7ff8000000000000ull;
            es = 8;
            std::memcpy(nan, &v, 8);
        } else if (h->dtype == HLBM_F32) {
            const uint32_t v = 0x7fc00000u;
            es = 4;
            std::memcpy(nan, &v, 4);
        } else {
            const uint16_t v = h->dtype == HLBM_F16 ? 0x7e00u : 0x7fc0u;
            es = 2;
            std::memcpy(nan, &v, 2);
        }
        cudaError_t e = cudaSuccess;
        for (int i = 0; i < 9 && e == cudaSuccess; ++i)
            e = cudaMemcpyAsync((unsigned char*)h->fbuf[h->fi] + es * (size_t)(i * plane + y * pitch + x), nan, es,
                                cudaMemcpyHostToDevice, h->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
        return cuda_check(h, e, "NaN injection");
    }
    return fail(h, HLBM_EINVAL, "unknown fault kind %d", (int)kind);
}

int hlbm_status(hlbm_t* h, uint32_t* bits) {
    if (!h || !bits) return HLBM_EINVAL;
    unsigned v = 0;
    int rc = sync_status(h, &v);
    *bits = v;
    return rc;
}

int hlbm_force(hlbm_t* h, int64_t first, int64_t count, double* fx, double* fy) {
    if (!h || first < 0 || count < 0 || first + count > h->t + 1) return HLBM_EINVAL;
    std::vector<double> buf(2 * (size_t)count);
    cudaError_t e = cudaMemcpyAsync(buf.data(), h->force + 2 * first, 2 * (size_t)count * sizeof(double),
                                    cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_check(h, e, "force readback");
    for (int64_t k = 0; k < count; ++k) {
        if (fx) fx[k] = buf[2 * k];
        if (fy) fy[k] = buf[2 * k + 1];
    }
    unsigned st;
    int rc = sync_status(h, &st);
    if (rc != HLBM_OK) return rc;
    return status_error(h, st);
}

namespace {
// Theta from the fit of the force history over the steps t0..t1 (Sec. 2.1)
int theta_window(hlbm* h, int64_t t0, int64_t t1, double* re, double* im, double* rms) {
    const double PI = 3.14159265358979323846;
    if (t1 > h->t || t1 <= t0 || t0 < 0)
        return fail(h, HLBM_EINVAL, "fit window [%lld, %lld] is not inside the %lld steps taken", (long long)t0,
                    (long long)t1, (long long)h->t);
    launch_gamma_sums(h->force, t0, t1, h->motion.omega, h->scratch, h->stream);
    double sums[5];
    cudaError_t e = cudaMemcpyAsync(sums, h->scratch, sizeof sums, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_check(h, e, "fit readback");
    double det = sums[0] * sums[2] - sums[1] * sums[1];
    double a = (sums[3] * sums[2] - sums[4] * sums[1]) / det;
    double b = (sums[4] * sums[0] - sums[3] * sums[1]) / det;
    launch_gamma_resid(h->force, t0, t1, h->motion.omega, a, b, h->scratch + 8, h->stream);
    double r2 = 0;
    e = cudaMemcpyAsync(&r2, h->scratch + 8, sizeof r2, cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_check(h, e, "fit readback");
    double N = 0.25 * PI * h->grid.rho0 * h->motion.omega * h->motion.omega * h->patch.lamina_L *
               h->patch.lamina_L * h->motion.A;
    *re = a / N;
    *im = b / N;
    if (rms) *rms = std::sqrt(r2 / (double)(t1 - t0 + 1)) / N;
    unsigned st;
    int rc = sync_status(h, &st);
    if (rc != HLBM_OK) return rc;
    return status_error(h, st);
}
}  // namespace

int hlbm_gamma(hlbm_t* h, double discard_periods, double fit_periods, double* re, double* im, double* rms) {
    if (!h || !re || !im) return HLBM_EINVAL;
    if (h->motion.kind != HLBM_MOTION_HARMONIC || !(h->motion.omega > 0) || h->motion.A == 0.0)
        return fail(h, HLBM_EINVAL, "the hydrodynamic function needs harmonic motion");
    const double PI = 3.14159265358979323846;
    double Tp = 2.0 * PI / h->motion.omega;
    int64_t t0 = (int64_t)std::ceil(discard_periods * Tp);
    int64_t t1 = (int64_t)std::floor((discard_periods + fit_periods) * Tp);
    return theta_window(h, t0, t1, re, im, rms);
}

int hlbm_theta_gradient(const hlbm_grid_t* grid, const hlbm_patch_t* patch, double tau_s,
                        const hlbm_motion_t* motion, int64_t nsteps, double discard_periods, double fit_periods,
                        double rel_step, void* cuda_stream, double* theta, double* grad, double* sweep_ms) {
    std::string& err = g_create_err;
    if (!grid || !patch || !motion || !theta || !grad || nsteps < 1 || !(rel_step > 0.0) || !(rel_step < 0.1)) {
        err = "hlbm_theta_gradient: invalid argument";
        return HLBM_EINVAL;
    }
    if (motion->kind != HLBM_MOTION_HARMONIC || !(motion->omega > 0) || motion->A == 0.0) {
        err = "hlbm_theta_gradient: the hydrodynamic function needs harmonic motion";
        return HLBM_EINVAL;
    }
    // the base point and (A, omega, tau_s) each moved by -/+ rel_step of their value
    const double base[3] = {motion->A, motion->omega, tau_s};
    double step[3];
    for (int k = 0; k < 3; ++k) step[k] = rel_step * std::fabs(base[k]);
    std::vector<hlbm*> inst(7, nullptr);
    int rc = HLBM_OK;
    for (int i = 0; i < 7 && rc == HLBM_OK; ++i) {
        hlbm_motion_t m = *motion;
        double ts = tau_s;
        if (i > 0) {
            const int k = (i - 1) / 2;
            const double dp = (i % 2 == 1 ? -1.0 : 1.0) * step[k];
            if (k == 0) m.A += dp;
            if (k == 1) m.omega += dp;
            if (k == 2) ts += dp;
        }
        rc = hlbm_create(grid, patch, ts, &m, cuda_stream, &inst[i]);
    }
    hlbm_sweep* w = nullptr;
    if (rc == HLBM_OK) rc = hlbm_sweep_create(7, inst.data(), cuda_stream, &w);
    if (rc == HLBM_OK) {
        rc = hlbm_sweep_pack(w, 1, nullptr);
        if (rc != HLBM_OK) err = w->err;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (rc == HLBM_OK && sweep_ms) {
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        cudaEventRecord(e0, (cudaStream_t)cuda_stream);
    }
    if (rc == HLBM_OK) {
        rc = hlbm_sweep_step(w, nsteps);
        if (rc != HLBM_OK) err = w->err;
    }
    if (rc == HLBM_OK && sweep_ms) {
        cudaEventRecord(e1, (cudaStream_t)cuda_stream);
        cudaEventSynchronize(e1);
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        *sweep_ms = ms;
    }
    // one fit window for all seven runs, in steps of the base period
    const double PI = 3.14159265358979323846;
    const double Tp = 2.0 * PI / motion->omega;
    const int64_t t0 = (int64_t)std::ceil(discard_periods * Tp);
    const int64_t t1 = (int64_t)std::floor((discard_periods + fit_periods) * Tp);
    double re[7] = {0}, im[7] = {0};
    for (int i = 0; i < 7 && rc == HLBM_OK; ++i) {
        rc = theta_window(inst[i], t0, t1, &re[i], &im[i], nullptr);
        if (rc != HLBM_OK) err = inst[i]->err;
    }
    if (rc == HLBM_OK) {
        theta[0] = re[0];
        theta[1] = im[0];
        for (int k = 0; k < 3; ++k) {
            grad[2 * k] = (re[2 + 2 * k] - re[1 + 2 * k]) / (2.0 * step[k]);
            grad[2 * k + 1] = (im[2 + 2 * k] - im[1 + 2 * k]) / (2.0 * step[k]);
        }
    } else if (err.empty()) {
        err = "hlbm_theta_gradient failed";
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (w) hlbm_sweep_destroy(w);
    for (hlbm* h : inst)
        if (h) hlbm_destroy(h);
    return rc;
}

int hlbm_theta_adjoint(const hlbm_grid_t* grid, const hlbm_patch_t* patch, double tau_s, const hlbm_motion_t* motion,
                       int64_t nsteps, double discard_periods, double fit_periods, double w_re, double w_im,
                       int32_t checkpoint_every, void* cuda_stream, double* theta, double* grad, double* fwd_ms,
                       double* bwd_ms) {
    std::string& err = g_create_err;
    if (!grid || !patch || !motion || !theta || !grad || nsteps < 1 || checkpoint_every < 1) {
        err = "hlbm_theta_adjoint: invalid argument";
        return HLBM_EINVAL;
    }
    if (motion->kind != HLBM_MOTION_HARMONIC || !(motion->omega > 0) || motion->A == 0.0 || grid->n_levels != 0 ||
        patch->outer_fv != 0 || grid->sponge_rows != 0 || (grid->dtype != HLBM_F64 && grid->dtype != HLBM_F32)) {
        err = "hlbm_theta_adjoint: needs HARMONIC motion, one lattice level, outer_fv = 0, no absorbing layer and "
              "FP64 or FP32";
        return HLBM_EINVAL;
    }
    hlbm_t* h = nullptr;
    int rc = hlbm_create(grid, patch, tau_s, motion, cuda_stream, &h);
    if (rc != HLBM_OK) return rc;
    rc = h->dtype == HLBM_F64 ? adjoint_impl<double>(h, nsteps, discard_periods, fit_periods, w_re, w_im,
                                                     checkpoint_every, theta, grad, fwd_ms, bwd_ms)
                              : adjoint_impl<float>(h, nsteps, discard_periods, fit_periods, w_re, w_im,
                                                    checkpoint_every, theta, grad, fwd_ms, bwd_ms);
    if (rc != HLBM_OK) err = "hlbm_theta_adjoint: " + h->err;
    hlbm_destroy(h);
    return rc;
}

int hlbm_get_fields(hlbm_t* h, double* rho_s, double* ux_s, double* uy_s, double* rho_u, double* ux_u,
                    double* uy_u) {
    if (!h) return HLBM_EINVAL;
    int rc = HLBM_OK;
    const size_t N = (size_t)h->grid.nx * h->grid.ny, n = h->patch.n_nodes;
    double* buf = (double*)dev_alloc(h, (3 * N + 3 * n) * sizeof(double));
    if (!buf) return fail(h, HLBM_ENOMEM, "readback buffer");
    if (h->dtype != HLBM_F64) {
        bind(h, h->df);
        launch_struct_macro<float>(h->df, buf, buf + N, buf + 2 * N, h->stream);
        launch_patch_macro<float>(h->df, buf + 3 * N, buf + 3 * N + n, buf + 3 * N + 2 * n, nullptr, h->stream);
    } else {
        bind(h, h->dd);
        launch_struct_macro<double>(h->dd, buf, buf + N, buf + 2 * N, h->stream);
        launch_patch_macro<double>(h->dd, buf + 3 * N, buf + 3 * N + n, buf + 3 * N + 2 * n, nullptr, h->stream);
    }
    double* dst[3] = {rho_s, ux_s, uy_s};
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 3 && e == cudaSuccess; ++k)
        if (dst[k]) e = cudaMemcpyAsync(dst[k], buf + k * N, N * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    std::vector<double> patch(3 * n);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(patch.data(), buf + 3 * N, 3 * n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) rc = cuda_check(h, e, "field readback");
    double* pdst[3] = {rho_u, ux_u, uy_u};
    for (int k = 0; k < 3 && rc == HLBM_OK; ++k)
        if (pdst[k])
            for (size_t p = 0; p < n; ++p) pdst[k][h->perm[p]] = patch[k * n + p];
    dev_free(h, buf);
    return rc;
}

int hlbm_get_level_fields(hlbm_t* h, int32_t level, double* rho, double* ux, double* uy) {
    if (!h) return HLBM_EINVAL;
    if (level < 1 || level > (int)h->lv.size())
        return fail(h, HLBM_EINVAL, "level %d: the solver has %zu coarser levels", level, h->lv.size());
    hlbm::Level& L = h->lv[level - 1];
    const size_t N = (size_t)L.ref.nxc * L.ref.nyc;
    double* buf = (double*)dev_alloc(h, 3 * N * sizeof(double));
    if (!buf) return fail(h, HLBM_ENOMEM, "readback buffer");
    if (h->dtype != HLBM_F64) {
        L.df.fA = (float*)L.buf[L.cur];
        launch_struct_macro<float>(L.df, buf, buf + N, buf + 2 * N, h->stream);
    } else {
        L.dd.fA = (double*)L.buf[L.cur];
        launch_struct_macro<double>(L.dd, buf, buf + N, buf + 2 * N, h->stream);
    }
    double* dst[3] = {rho, ux, uy};
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < 3 && e == cudaSuccess; ++k)
        if (dst[k]) e = cudaMemcpyAsync(dst[k], buf + k * N, N * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    int rc = e == cudaSuccess ? HLBM_OK : cuda_check(h, e, "level field readback");
    dev_free(h, buf);
    return rc;
}

int hlbm_get_patch_f(hlbm_t* h, double* f9) {
    if (!h || !f9) return HLBM_EINVAL;
    const size_t n = h->patch.n_nodes;
    double* buf = (double*)dev_alloc(h, 9 * n * sizeof(double));
    if (!buf) return fail(h, HLBM_ENOMEM, "readback buffer");
    if (h->dtype != HLBM_F64) {
        bind(h, h->df);
        launch_patch_macro<float>(h->df, nullptr, nullptr, nullptr, buf, h->stream);
    } else {
        bind(h, h->dd);
        launch_patch_macro<double>(h->dd, nullptr, nullptr, nullptr, buf, h->stream);
    }
    std::vector<double> tmp(9 * n);
    cudaError_t e = cudaMemcpyAsync(tmp.data(), buf, 9 * n * sizeof(double), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    dev_free(h, buf);
    if (e != cudaSuccess) return cuda_check(h, e, "patch readback");
    for (size_t p = 0; p < n; ++p)
        for (int i = 0; i < 9; ++i) f9[9 * (size_t)h->perm[p] + i] = tmp[9 * p + i];
    return HLBM_OK;
}

int hlbm_get_class(hlbm_t* h, int8_t* cls) {
    if (!h || !cls) return HLBM_EINVAL;
    const int bw = h->dtype != HLBM_F64 ? h->df.bw : h->dd.bw;
    const int bh = h->dtype != HLBM_F64 ? h->df.bh : h->dd.bh;
    std::vector<int8_t> win((size_t)bw * bh);
    cudaError_t e = cudaMemcpyAsync(win.data(), h->cls[h->ci], win.size(), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_check(h, e, "class readback");
    const int nx = h->grid.nx, ny = h->grid.ny;
    std::memset(cls, CLS_DISC, (size_t)nx * ny);
    for (int j = 0; j < bh; ++j)
        for (int i = 0; i < bw; ++i) {
            int x = h->pbx0 + i, y = h->pby0 + j;
            if (x >= 0 && y >= 0 && x < nx && y < ny) cls[(size_t)y * nx + x] = win[(size_t)j * bw + i];
        }
    return HLBM_OK;
}

int hlbm_get_refill(hlbm_t* h, int32_t* type, int32_t* donor) {
    if (!h) return HLBM_EINVAL;
    const size_t n = h->patch.n_nodes;
    int32_t* rt = h->dtype != HLBM_F64 ? h->df.rtype : h->dd.rtype;
    int32_t* rd = h->dtype != HLBM_F64 ? h->df.rdonor : h->dd.rdonor;
    std::vector<int32_t> t(n), d(n);
    cudaError_t e = cudaMemcpyAsync(t.data(), rt, n * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(d.data(), rd, n * sizeof(int32_t), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_check(h, e, "refill readback");
    for (size_t p = 0; p < n; ++p) {
        if (type) type[h->perm[p]] = t[p];
        if (donor) donor[h->perm[p]] = d[p];
    }
    return HLBM_OK;
}

int hlbm_get_fv(hlbm_t* h, int32_t* row_ptr, int32_t* col, double* gx, double* gy, double* cc) {
    if (!h) return HLBM_EINVAL;
    return h->dtype != HLBM_F64 ? get_fv_impl<float>(h, h->df.coef, row_ptr, col, gx, gy, cc)
                                : get_fv_impl<double>(h, h->dd.coef, row_ptr, col, gx, gy, cc);
}

int hlbm_info(hlbm_t* h, hlbm_info_t* info) {
    if (!h || !info) return HLBM_EINVAL;
    const int bw = h->dtype != HLBM_F64 ? h->df.bw : h->dd.bw;
    const int bh = h->dtype != HLBM_F64 ? h->df.bh : h->dd.bh;
    std::vector<int8_t> win((size_t)bw * bh);
    cudaError_t e = cudaMemcpyAsync(win.data(), h->cls[h->ci], win.size(), cudaMemcpyDeviceToHost, h->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
    if (e != cudaSuccess) return cuda_check(h, e, "class readback");
    int64_t nondisc = 0;
    for (int8_t c : win) nondisc += (c != CLS_DISC);
    info->time = h->t;
    info->n_struct = (int64_t)h->grid.nx * h->grid.ny;
    info->n_struct_disc = info->n_struct - nondisc;
    info->n_nodes = h->patch.n_nodes;
    info->n_tris = h->patch.n_tris;
    info->nnz = h->nnz;
    info->n_outer = (int32_t)h->outer.size();
    info->n_wall_segments = h->nseg;
    info->box_w = bw;
    info->box_h = bh;
    // refill, classify, fill, stream-collide, feed, FV sub-steps, force (2)
    // with levels: + one coupling launch and one stream-collide per level
    // at a step where all of them start (every 2^n_levels steps)
    info->launches_per_step = 8 + 2 * (int32_t)h->lv.size();
    info->n_levels = (int32_t)h->lv.size();
    info->n_coarse = 0;
    info->coarse_updates = 0.0;
    for (size_t k = 0; k < h->lv.size(); ++k) {
        const int64_t nk = (int64_t)h->lv[k].ref.nxc * h->lv[k].ref.nyc;
        info->n_coarse += nk;
        info->coarse_updates += std::ldexp((double)nk, -(int)(k + 1));
    }
    info->fv_kernel = h->fv_kind;
    info->n_tiles = h->n_tiles;
    info->fv_depth = 1;
    info->fv_slots = 0;
    if (h->fv_kind == HLBM_FV_DEEP) {
        info->fv_depth = h->dtype != HLBM_F64 ? h->df.deep_k : h->dd.deep_k;
        info->fv_slots = h->dtype != HLBM_F64 ? h->df.deep_slot_cap : h->dd.deep_slot_cap;
    }
    if (h->motion.kind == HLBM_MOTION_INDUCED) {
        info->y = h->Yi;
        info->vy = h->Vi;
    } else {
        double X, Y;
        motion_pos(h->motion, h->t, &X, &Y);
        info->y = Y;
        info->vy = h->motion.kind == HLBM_MOTION_HARMONIC
                       ? h->motion.A * h->motion.omega * std::cos(h->motion.omega * (double)h->t)
                       : h->motion.kind == HLBM_MOTION_UNIFORM ? h->motion.vy : 0.0;
    }
    info->dtype = h->dtype;
    return HLBM_OK;
}

int hlbm_profile(hlbm_t* h, int enable) {
    if (!h) return HLBM_EINVAL;
    int rc = phase_collect(h);
    if (rc != HLBM_OK) return rc;
    h->profiling = enable != 0;
    if (enable)
        for (int k = 0; k < HLBM_N_PHASES; ++k) {
            h->phase_ms[k] = 0.0;
            h->phase_launches[k] = 0;
        }
    return HLBM_OK;
}

int hlbm_profile_read(hlbm_t* h, double* ms, int64_t* launches) {
    if (!h) return HLBM_EINVAL;
    int rc = phase_collect(h);
    if (rc != HLBM_OK) return rc;
    for (int k = 0; k < HLBM_N_PHASES; ++k) {
        if (ms) ms[k] = h->phase_ms[k];
        if (launches) launches[k] = h->phase_launches[k];
    }
    return HLBM_OK;
}

int hlbm_sweep_create(int32_t n, hlbm_t* const* solvers, void* cuda_stream, hlbm_sweep_t** out) {
    if (!out || n < 1 || !solvers) return HLBM_EINVAL;
    *out = nullptr;
    for (int i = 0; i < n; ++i)
        if (!solvers[i]) return HLBM_EINVAL;
    hlbm_sweep* w = new hlbm_sweep();
    w->main = (cudaStream_t)cuda_stream;
    w->inst.assign(solvers, solvers + n);
    w->streams.resize(n);
    w->ev_lat.resize(n);
    w->ev_fv.resize(n);
    w->ev_done.resize(n);
    w->fv_t0.resize(n);
    w->fv_t1.resize(n);
    w->fv_ms.assign(n, 0.0);
    w->tile_nodes.assign(n, 0);
    bool ok = cudaStreamCreateWithFlags(&w->fv, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&w->ev_main, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; i < n && ok; ++i) {
        ok = cudaStreamCreateWithFlags(&w->streams[i], cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreateWithFlags(&w->ev_lat[i], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&w->ev_fv[i], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreateWithFlags(&w->ev_done[i], cudaEventDisableTiming) == cudaSuccess &&
             cudaEventCreate(&w->fv_t0[i]) == cudaSuccess && cudaEventCreate(&w->fv_t1[i]) == cudaSuccess;
    }
    if (!ok) {
        hlbm_sweep_destroy(w);
        return HLBM_ECUDA;
    }
    *out = w;
    return HLBM_OK;
}

// every stream of the sweep waits for the work already queued on `from`,
// and instance i's stream also for the work queued on that solver's own stream
static void sweep_fork(hlbm_sweep* w, cudaStream_t from) {
    cudaEventRecord(w->ev_main, from);
    cudaStreamWaitEvent(w->fv, w->ev_main, 0);
    for (size_t i = 0; i < w->inst.size(); ++i) {
        cudaStreamWaitEvent(w->streams[i], w->ev_main, 0);
        if (w->inst[i]->stream != from) {
            cudaEventRecord(w->ev_done[i], w->inst[i]->stream);
            cudaStreamWaitEvent(w->streams[i], w->ev_done[i], 0);
        }
    }
}

// `to` and every instance's own stream wait for all the sweep's work
static void sweep_join(hlbm_sweep* w, cudaStream_t to) {
    for (size_t i = 0; i < w->inst.size(); ++i) {
        cudaEventRecord(w->ev_done[i], w->streams[i]);
        cudaStreamWaitEvent(to, w->ev_done[i], 0);
        if (w->inst[i]->stream != to) cudaStreamWaitEvent(w->inst[i]->stream, w->ev_done[i], 0);
    }
    cudaEventRecord(w->ev_main, w->fv);
    cudaStreamWaitEvent(to, w->ev_main, 0);
}

// an instance with status bits the host has seen refuses to be stepped, as
// in hlbm_step
static int sweep_check(hlbm_sweep* w) {
    for (size_t i = 0; i < w->inst.size(); ++i) {
        int rc = check_fault(w->inst[i]);
        if (rc != HLBM_OK) {
            w->err = "instance " + std::to_string(i) + ": " + w->inst[i]->err;
            return rc;
        }
    }
    return HLBM_OK;
}

int hlbm_sweep_step(hlbm_sweep_t* w, int64_t nsteps) {
    if (!w || nsteps < 0) return HLBM_EINVAL;
    int rc = sweep_check(w);
    if (rc != HLBM_OK) return rc;
    sweep_fork(w, w->main);
    for (int64_t k = 0; k < nsteps && rc == HLBM_OK; ++k) rc = sweep_one_step(w, false);
    sweep_join(w, w->main);
    if (nsteps > 0)
        for (hlbm* h : w->inst) queue_status_copy(h);
    return rc;
}

int hlbm_sweep_tune(hlbm_sweep_t* w, int32_t trial_steps, int32_t* tile_nodes) {
    if (!w || trial_steps < 1) return HLBM_EINVAL;
    if (int rc = sweep_check(w); rc != HLBM_OK) return rc;
    // the tuner times every solver's own launch: no packs
    for (cudaEvent_t e : w->ev_pack)
        if (e) cudaEventDestroy(e);
    w->ev_pack.clear();
    w->packs.clear();
    w->pack_of.assign(w->inst.size(), -1);
    const int candidates[] = {256, 512, 1024, 1536};
    const size_t n = w->inst.size();
    std::vector<double> best(n, 1e300);
    std::vector<int32_t> pick(n, 0);
    int rc = HLBM_OK;
    for (int c : candidates) {
        for (size_t i = 0; i < n && rc == HLBM_OK; ++i) {
            const int nodes = w->inst[i]->patch.n_nodes;
            rc = inst_retile(w->inst[i], (nodes + c - 1) / c);
        }
        if (rc != HLBM_OK) break;
        std::fill(w->fv_ms.begin(), w->fv_ms.end(), 0.0);
        sweep_fork(w, w->main);
        for (int32_t k = 0; k < trial_steps && rc == HLBM_OK; ++k) rc = sweep_one_step(w, true);
        sweep_join(w, w->main);
        for (size_t i = 0; i < n; ++i)
            if (w->fv_ms[i] < best[i]) {
                best[i] = w->fv_ms[i];
                pick[i] = c;
            }
    }
    for (size_t i = 0; i < n && rc == HLBM_OK; ++i) {
        const int nodes = w->inst[i]->patch.n_nodes;
        rc = inst_retile(w->inst[i], (nodes + pick[i] - 1) / pick[i]);
        w->tile_nodes[i] = pick[i];
        if (tile_nodes) tile_nodes[i] = pick[i];
    }
    cudaStreamSynchronize(w->main);
    return rc;
}

int hlbm_sweep_fv_time(hlbm_sweep_t* w, int64_t nsteps, double* fv_ms) {
    if (!w || nsteps < 1 || !fv_ms) return HLBM_EINVAL;
    if (int rc = sweep_check(w); rc != HLBM_OK) return rc;
    std::fill(w->fv_ms.begin(), w->fv_ms.end(), 0.0);
    sweep_fork(w, w->main);
    int rc = HLBM_OK;
    for (int64_t k = 0; k < nsteps && rc == HLBM_OK; ++k) rc = sweep_one_step(w, true);
    sweep_join(w, w->main);
    for (size_t i = 0; i < w->inst.size(); ++i) fv_ms[i] = w->fv_ms[i];
    return rc;
}

int hlbm_sweep_pack(hlbm_sweep_t* w, int32_t enable, int32_t* n_packs) {
    if (!w) return HLBM_EINVAL;
    for (cudaEvent_t e : w->ev_pack)
        if (e) cudaEventDestroy(e);
    w->ev_pack.clear();
    w->packs.clear();
    const int n = (int)w->inst.size();
    w->pack_of.assign(n, -1);
    int rc = HLBM_OK;
    if (enable) {
        int sms = 0, dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        std::vector<int> order;
        for (int i = 0; i < n; ++i)
            if (w->inst[i]->patch.outer_fv == 0 && w->inst[i]->patch.fv_kernel == HLBM_FV_AUTO) order.push_back(i);
        std::sort(order.begin(), order.end(), [&](int a, int b) {
            const hlbm *ha = w->inst[a], *hb = w->inst[b];
            if ((ha->dtype == HLBM_F64) != (hb->dtype == HLBM_F64)) return ha->dtype != HLBM_F64;
            if (ha->patch.n_sub != hb->patch.n_sub) return ha->patch.n_sub < hb->patch.n_sub;
            return a < b;
        });
        auto tile_max = [](const hlbm* h) { return h->dtype != HLBM_F64 ? fv_tile_max<float>() : fv_tile_max<double>(); };
        auto min_tiles = [&](const hlbm* h) { return (h->patch.n_nodes + tile_max(h) - 1) / tile_max(h); };
        size_t k = 0;
        while (k < order.size() && rc == HLBM_OK) {
            // a group: same precision, sub-step counts within 25 %, at most
            // kFvPackMax solvers, one block per SM in all
            std::vector<int> g{order[k]};
            int need = min_tiles(w->inst[order[k]]);
            const hlbm* h0 = w->inst[order[k]];
            size_t j = k + 1;
            while (j < order.size()) {
                const hlbm* h = w->inst[order[j]];
                if ((h->dtype == HLBM_F64) != (h0->dtype == HLBM_F64) || h->patch.n_sub * 4 > h0->patch.n_sub * 5 ||
                    (int)g.size() >= kFvPackMax || need + min_tiles(h) > sms)
                    break;
                need += min_tiles(h);
                g.push_back(order[j]);
                ++j;
            }
            k = j;
            if (g.size() < 2) continue;
            // share the SMs in proportion to each solver's FV work
            double wsum = 0;
            for (int i : g) wsum += (double)w->inst[i]->patch.n_nodes * w->inst[i]->patch.n_sub;
            std::vector<int> tiles;
            int tsum = 0;
            for (int i : g) {
                const hlbm* h = w->inst[i];
                int t = (int)std::floor(sms * (double)h->patch.n_nodes * h->patch.n_sub / wsum);
                t = std::min(t, std::max(1, h->patch.n_nodes / 64));
                t = std::max(t, min_tiles(h));
                tiles.push_back(t);
                tsum += t;
            }
            while (tsum > sms) {
                size_t big = 0;
                for (size_t q = 0; q < g.size(); ++q)
                    if (tiles[q] - min_tiles(w->inst[g[q]]) > tiles[big] - min_tiles(w->inst[g[big]])) big = q;
                if (tiles[big] <= min_tiles(w->inst[g[big]])) break;
                --tiles[big];
                --tsum;
            }
            bool ok = tsum <= sms;
            for (size_t q = 0; q < g.size() && ok && rc == HLBM_OK; ++q) {
                hlbm* h = w->inst[g[q]];
                // tiles the tensor-memory kernel cannot hold (its shared
                // memory grows with the tile and its halo) are made smaller,
                // a quarter more tiles at a time, while the SMs last
                for (;;) {
                    rc = inst_retile(h, tiles[q], true);
                    if (rc != HLBM_EINVAL) break;
                    const int more = std::max(1, tiles[q] / 4);
                    if (tsum + more > sms || tiles[q] + more > std::max(1, h->patch.n_nodes / 64)) break;
                    tiles[q] += more;
                    tsum += more;
                }
                if (rc == HLBM_EINVAL) {
                    rc = HLBM_OK;
                    ok = false;
                    break;
                }
                ok = rc == HLBM_OK && h->fv_kind == HLBM_FV_TMEM && h->n_tiles == tiles[q];
            }
            if (rc != HLBM_OK) {
                w->err = "packing: " + w->inst[g[0]]->err;
                break;
            }
            if (!ok) {
                // this group stays unpacked, each solver with its own tiling
                for (int i : g) rc = rc == HLBM_OK ? inst_retile(w->inst[i], tuned_tiles(w, i)) : rc;
                if (rc != HLBM_OK) w->err = "packing: " + w->inst[g[0]]->err;
                continue;
            }
            cudaEvent_t e = nullptr;
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) {
                rc = HLBM_ECUDA;
                break;
            }
            w->ev_pack.push_back(e);
            for (int i : g) w->pack_of[i] = (int)w->packs.size();
            w->packs.push_back(g);
        }
    } else {
        for (int i = 0; i < n && rc == HLBM_OK; ++i) rc = inst_retile(w->inst[i], tuned_tiles(w, i));
    }
    if (n_packs) *n_packs = (int32_t)w->packs.size();
    return rc;
}

const char* hlbm_sweep_last_error(const hlbm_sweep_t* w) { return w ? w->err.c_str() : "null sweep"; }

void hlbm_sweep_destroy(hlbm_sweep_t* w) {
    if (!w) return;
    if (w->main) cudaStreamSynchronize(w->main);
    for (cudaStream_t s : w->streams)
        if (s) {
            cudaStreamSynchronize(s);
            cudaStreamDestroy(s);
        }
    if (w->fv) {
        cudaStreamSynchronize(w->fv);
        cudaStreamDestroy(w->fv);
    }
    for (auto* v : {&w->ev_lat, &w->ev_fv, &w->ev_done, &w->fv_t0, &w->fv_t1, &w->ev_pack})
        for (cudaEvent_t e : *v)
            if (e) cudaEventDestroy(e);
    if (w->ev_main) cudaEventDestroy(w->ev_main);
    delete w;
}

int hlbm_save(hlbm_t* h, const char* path) {
    if (!h || !path) return HLBM_EINVAL;
    return h->dtype != HLBM_F64 ? save_impl<float>(h, path) : save_impl<double>(h, path);
}

int hlbm_load(hlbm_t* h, const char* path) {
    if (!h || !path) return HLBM_EINVAL;
    h->far_ready = false;
    return h->dtype != HLBM_F64 ? load_impl<float>(h, path) : load_impl<double>(h, path);
}

const char* hlbm_last_error(const hlbm_t* h) { return h ? h->err.c_str() : g_create_err.c_str(); }

void hlbm_destroy(hlbm_t* h) {
    if (!h) return;
    cudaStreamSynchronize(h->stream);
    if (h->side) {
        cudaStreamSynchronize(h->side);
        cudaStreamDestroy(h->side);
    }
    for (cudaEvent_t e : {h->ev_fv, h->ev_force, h->ev_move, h->ev_cls})
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : h->ev_pool) cudaEventDestroy(e);
    if (h->st_event) cudaEventDestroy(h->st_event);
    if (h->st_host) cudaFreeHost(h->st_host);
    for (void* b : std::vector<void*>(h->blocks)) dev_free(h, b);
    delete h;
}

}  // extern "C"
