// emt_api.cu -- host runtime and C ABI (include/emt.h): device memory plan,
// table and geometry upload, event admission, the step-loop drivers
// (plain host loop and CUDA-graph replay) and score read-back.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>
#include <string>
#include <unordered_map>
#include <vector>

#include "../../include/emt.h"
#include "emt_internal.h"

using namespace emt;

namespace {

constexpr int kMaxGrid = 129;  // at most 128 intervals
constexpr size_t kAlign = 256;
// bound of one grid-barrier wait of the persistent step loop (a wait
// outlasts the slowest block's step; steps of the populations the
// persistent loop is meant for take milliseconds)
constexpr double kPersistWaitMs = 10000.0;

size_t align_up(size_t v) { return (v + kAlign - 1) / kAlign * kAlign; }

// Byte layout of every device buffer inside one pool.
struct Plan {
    size_t total = 0;
    size_t add(size_t bytes)
    {
        size_t off = total;
        total += align_up(bytes ? bytes : 1);
        return off;
    }
    // tracks: [side][field]
    size_t trk[2][11];
    size_t cnt, status, total_steps, done_head, ehist, gsync;
    size_t hist, ledger, counts, live, event_id, done_ring;
    size_t grid, gridf, igrid, igridf, irs, irsf, tab, tabf, dedx, mats, bk, vacuum, x0, ray_a, scratch;
    size_t dgrid, dgridf, dtab, dtabf;
    size_t zb, lmat, lbin;
    size_t st_ev, st_type, st_T, st_pos, st_dir, st_uid, st_slot, st_ids, st_start, st_runs;
    size_t slots_tmp, out_hist, out_summary;
    size_t iq[13];      // split schedule: interaction queue fields
    size_t iq_alt[13];  // pipelined schedule: the second queue
    size_t skey, sperm;  // split schedule: scheduling classes and order of charged tracks in a field
    size_t step_hist;  // [3][step_bins] when step_bins > 0
    int step_bins;
    size_t spill[11];     // host spill: staging buffer of Q track records (when spill_above > 0)
    size_t spill_ticket;  // [3]
    bool spill_on;
    int64_t Q;
    int max_events, hstride, max_prim;
    bool mixed;
    bool split;      // a queue of interacting tracks (split or pipelined schedule)
    bool pipelined;  // one kernel per step, interactions sampled one iteration later
};

Plan make_plan(const emt_options& o)
{
    Plan p;
    p.Q = o.slot_capacity;
    p.max_events = o.max_events;
    p.hstride = o.max_bins + 1;
    p.mixed = o.precision == EMT_PRECISION_MIXED;
    p.max_prim = (int)std::min<int64_t>(p.Q, 1 << 22);
    const size_t Q = (size_t)p.Q;
    const size_t rs = p.mixed ? 4 : 8;
    const size_t fs[11] = {8, 8, 8, rs, rs, rs, rs, 8, 4, 4, 4};
    for (int s = 0; s < 2; ++s)
        for (int f = 0; f < 11; ++f) p.trk[s][f] = p.add(Q * fs[f]);
    p.cnt = p.add(3 * sizeof(Counters));
    p.status = p.add(sizeof(int));
    p.total_steps = p.add(4 * sizeof(unsigned long long));
    p.done_head = p.add(sizeof(unsigned));
    p.ehist = p.add(3 * kEBins * sizeof(unsigned));
    p.gsync = p.add(sizeof(GridSync));
    const size_t E = (size_t)p.max_events;
    p.hist = p.add(E * p.hstride * sizeof(double));
    p.ledger = p.add(E * 3 * sizeof(double));
    p.counts = p.add(E * 2 * sizeof(unsigned long long));
    p.live = p.add(E * sizeof(int));
    p.event_id = p.add(E * sizeof(uint64_t));
    p.done_ring = p.add(E * sizeof(unsigned));
    p.grid = p.add(kMaxGrid * sizeof(double));
    p.gridf = p.add(kMaxGrid * sizeof(float));
    p.igrid = p.add(kMaxGrid * sizeof(double));
    p.igridf = p.add(kMaxGrid * sizeof(float));
    p.irs = p.add((size_t)kMaxMat * 3 * kMaxGrid * sizeof(double));
    p.irsf = p.add((size_t)kMaxMat * 3 * kMaxGrid * sizeof(float));
    p.tab = p.add((size_t)kMaxMat * 3 * kMaxGrid * kNq * sizeof(double));
    p.tabf = p.add((size_t)kMaxMat * 3 * kMaxGrid * kNq * sizeof(float));
    p.dgrid = p.add(kMaxGrid * sizeof(double));
    p.dgridf = p.add(kMaxGrid * sizeof(float));
    p.dtab = p.add((size_t)kMaxMat * 3 * kMaxGrid * kNq * sizeof(double));
    p.dtabf = p.add((size_t)kMaxMat * 3 * kMaxGrid * kNq * sizeof(float));
    p.dedx = p.add((size_t)kMaxMat * 3 * kMaxGrid * sizeof(double));
    p.mats = p.add(kMaxMat * sizeof(MaterialDev));
    p.bk = p.add(kMaxMat * sizeof(double));
    p.vacuum = p.add(kMaxMat * sizeof(int));
    p.x0 = p.add(kMaxMat * sizeof(double));
    p.ray_a = p.add(kMaxMat * sizeof(double));
    p.scratch = p.add((32 + (size_t)kMaxMat * 2 * kMaxGrid) * sizeof(double));
    p.zb = p.add((kMaxLayers + 1) * sizeof(double));
    p.lmat = p.add(kMaxLayers * sizeof(int));
    p.lbin = p.add(kMaxLayers * sizeof(int));
    const size_t P = (size_t)p.max_prim;
    p.st_ev = p.add(P * 4);
    p.st_type = p.add(P * 4);
    p.st_T = p.add(P * 8);
    p.st_pos = p.add(P * 24);
    p.st_dir = p.add(P * 24);
    p.st_uid = p.add(P * 4);
    p.st_slot = p.add(E * 4);
    p.st_ids = p.add(E * 8);
    p.st_start = p.add(E * 4);
    p.st_runs = p.add(E * 4);
    p.slots_tmp = p.add(E * 4);
    p.split = o.schedule == EMT_SCHEDULE_SPLIT || o.schedule == EMT_SCHEDULE_PIPELINED;
    p.pipelined = o.schedule == EMT_SCHEDULE_PIPELINED;
    for (int f = 0; f < 13; ++f) p.iq_alt[f] = 0;
    if (p.split) {
        // x y z ux uy uz T uid dep ev step tv src
        const size_t iqs[13] = {8, 8, 8, rs, rs, rs, rs, 8, 8, 4, 4, 4, 4};
        for (int f = 0; f < 13; ++f) p.iq[f] = p.add(Q * iqs[f]);
        if (p.pipelined)
            for (int f = 0; f < 13; ++f) p.iq_alt[f] = p.add(Q * iqs[f]);
        p.skey = p.add(Q);
        p.sperm = p.add(Q * 4);
    } else {
        for (int f = 0; f < 13; ++f) p.iq[f] = 0;
        p.skey = p.sperm = 0;
    }
    p.out_hist = p.add(E * (size_t)o.max_bins * sizeof(double));
    p.out_summary = p.add(E * EMT_SUMMARY_LEN * sizeof(double));
    p.step_bins = o.step_hist_bins;
    p.step_hist = p.step_bins > 0 ? p.add((size_t)3 * p.step_bins * sizeof(unsigned long long)) : 0;
    p.spill_on = o.spill_above > 0;
    for (int f = 0; f < 11; ++f) p.spill[f] = p.spill_on ? p.add(Q * fs[f]) : 0;
    p.spill_ticket = p.add(3 * sizeof(int));
    return p;
}

bool valid_options(const emt_options& o, std::string& why)
{
    if (o.precision != EMT_PRECISION_FP64 && o.precision != EMT_PRECISION_MIXED) return why = "precision", false;
    if (o.slot_capacity < 64 || o.slot_capacity > (int64_t)1 << 30) return why = "slot_capacity out of [64, 2^30]", false;
    if (o.max_events < 1 || o.max_events > (1 << 24)) return why = "max_events out of [1, 2^24]", false;
    if (o.max_bins < 1 || o.max_bins > 65536) return why = "max_bins out of [1, 65536]", false;
    if (o.block_size != 0 && o.block_size != 128 && o.block_size != 256)
        return why = "block_size must be 0 (default), 128 or 256", false;
    if (o.loop_mode != EMT_LOOP_PLAIN && o.loop_mode != EMT_LOOP_GRAPH && o.loop_mode != EMT_LOOP_PERSISTENT)
        return why = "loop_mode", false;
    if (o.loop_mode == EMT_LOOP_PERSISTENT && o.graph_steps <= 0)
        return why = "graph_steps (steps per persistent launch) must be positive", false;
    if (o.schedule != EMT_SCHEDULE_FUSED && o.schedule != EMT_SCHEDULE_SPLIT && o.schedule != EMT_SCHEDULE_PIPELINED)
        return why = "schedule", false;
    if (o.loop_mode == EMT_LOOP_GRAPH && (o.graph_steps <= 0 || o.graph_steps % 6 != 0))
        return why = "graph_steps must be a positive multiple of 6", false;
    if (o.step_hist_bins < 0 || o.step_hist_bins > (1 << 20)) return why = "step_hist_bins out of [0, 2^20]", false;
    if (o.max_active < 0) return why = "max_active must be >= 0", false;
    if (o.select_policy != EMT_SELECT_ORDER && o.select_policy != EMT_SELECT_LOW_ENERGY)
        return why = "select_policy", false;
    if (o.max_active > 0 && o.schedule != EMT_SCHEDULE_SPLIT)
        return why = "track selection (max_active > 0) needs the split schedule", false;
    if (o.spill_above < 0) return why = "spill_above must be >= 0", false;
    if (o.spill_above > 0 &&
        (o.max_active <= 0 || o.select_policy != EMT_SELECT_LOW_ENERGY || o.spill_above < o.max_active))
        return why = "host spill needs low-energy track selection with spill_above >= max_active", false;
    return true;
}

// Validate a geometry description and lay out its arrays: zb[n + 1] (plane
// positions or shell radii), lm[n] (materials), lb[n] (score bins).
// Returns an error message, or nullptr.
const char* check_geometry(const emt_layer* layers, int n, const emt_world* w, int n_mat, int max_bins, double* zb,
                           int* lm, int* lb)
{
    if (n < 1 || n > kMaxLayers) return "layer count out of [1, 4096]";
    if (w->n_bins < 1 || w->n_bins > max_bins) return "n_bins out of [1, max_bins]";
    if (w->max_steps < 1) return "max_steps";
    if (w->geometry != EMT_GEOM_LAYERS && w->geometry != EMT_GEOM_CYLINDERS) return "geometry kind";
    if (w->score_z != 0 && w->score_z != 1) return "score_z must be 0 or 1";
    if (w->score_z && !(w->score_z_hi_cm > w->score_z_lo_cm)) return "score_z range must be non-empty";
    zb[0] = w->z0_cm;
    for (int i = 0; i < n; ++i) {
        if (!(layers[i].thickness_cm > 0.0)) return "layer thickness must be positive";
        if (layers[i].material < -1 || layers[i].material >= n_mat) return "layer material index";
        zb[i + 1] = zb[i] + layers[i].thickness_cm;
        lm[i] = layers[i].material;
        lb[i] = layers[i].score_bin;
    }
    if (w->geometry == EMT_GEOM_LAYERS) {
        if (!(w->half_x_cm > 0.0) || !(w->half_y_cm > 0.0)) return "stack half widths";
        const double lo[3] = {-w->half_x_cm, -w->half_y_cm, zb[0]};
        const double hi[3] = {w->half_x_cm, w->half_y_cm, zb[n]};
        for (int a = 0; a < 3; ++a)
            if (!(w->lo_cm[a] <= lo[a]) || !(w->hi_cm[a] >= hi[a])) return "the world box must contain the layer stack";
    } else {
        if (w->z0_cm != 0.0) return "cylinders: z0 (the innermost radius) must be 0";
        if (!(w->half_z_cm > 0.0)) return "cylinders: half_z must be positive";
    }
    const double b2 = w->B_tesla[0] * w->B_tesla[0] + w->B_tesla[1] * w->B_tesla[1] + w->B_tesla[2] * w->B_tesla[2];
    if (b2 > 0.0 && (!(w->rk_delta_cm > 0.0) || !(w->max_field_step_cm > 0.0)))
        return "field needs rk_delta_cm > 0 and max_field_step_cm > 0";
    return nullptr;
}

// geometry, field and scoring fields of the kernel parameters
template <typename R>
void set_geometry(Params<R>& p, int n, const emt_world* w)
{
    p.geom = w->geometry;
    p.half_z = w->half_z_cm;
    p.n_layers = n;
    p.hx = w->half_x_cm;
    p.hy = w->half_y_cm;
    p.kxy[0] = ord_key(-p.hx + kChordMargin);
    p.kxy[1] = ord_key(p.hx - kChordMargin);
    p.kxy[2] = ord_key(-p.hy + kChordMargin);
    p.kxy[3] = ord_key(p.hy - kChordMargin);
    for (int a = 0; a < 3; ++a) {
        p.wlo[a] = w->lo_cm[a];
        p.whi[a] = w->hi_cm[a];
        p.B[a] = w->B_tesla[a];
    }
    p.bmag = std::sqrt(w->B_tesla[0] * w->B_tesla[0] + w->B_tesla[1] * w->B_tesla[1] + w->B_tesla[2] * w->B_tesla[2]);
    p.rk_delta = w->rk_delta_cm;
    p.max_field_step = w->max_field_step_cm;
    p.has_field = p.bmag > 0.0 ? 1 : 0;
    p.max_steps = w->max_steps;
    p.n_bins = w->n_bins;
    p.score_z = w->score_z;
    p.zs_lo = w->score_z_lo_cm;
    p.zs_scale = w->score_z ? (double)w->n_bins / (w->score_z_hi_cm - w->score_z_lo_cm) : 1.0;
}

}  // namespace

struct emt_ctx {
    emt_options opt;
    Plan plan;
    std::string err;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    char* pool = nullptr;
    bool own_pool = false;
    bool poisoned = false;
    bool have_materials = false, have_geometry = false;
    int n_mat = 0, n_grid = 0, n_layers = 0, n_bins = 0;
    Params<double> pd;
    Params<float> pf;
    int64_t it = 0;  // step-loop iterations so far
    int64_t live_g = 0, live_c = 0;
    int64_t live_q = 0;  // pipelined schedule: interactions queued for the next iteration
    int resident_blocks = 0;
    int resident_a = 0, resident_b = 0;  // split schedule: transport, interaction kernels
    int persist_grid = 0;                // persistent step loop: resident blocks of the cooperative launch
    int resident_p = 0;                  // pipelined schedule: resident blocks of the step kernel
    long long wait_cycles = 0;           // bound of one grid-barrier wait, SM clock cycles
    int block = 128;
    // host event table
    std::vector<uint64_t> slot_id;
    std::vector<int> slot_state;  // 0 free, 1 in flight, 2 finished
    std::vector<int> free_slots;
    std::unordered_map<uint64_t, int> id_to_slot;
    std::vector<int> order;  // slots in submission order
    unsigned done_seen = 0;
    // host mirrors valid while no device work has run since they were read
    unsigned long long steps_seen[4] = {0, 0, 0, 0};  // total step, deferred, held and RK4-substep counters
    unsigned head_cached = 0;                    // finished-event ring head
    bool head_fresh = false;
    // pinned host mirrors
    Counters* h_cnt = nullptr;
    int* h_status = nullptr;
    unsigned long long* h_steps = nullptr;
    unsigned* h_done = nullptr;
    char* h_misc = nullptr;  // status .. done_head, read in one copy
    // CUDA graph of graph_steps iterations
    cudaGraphExec_t graph = nullptr;
    cudaEvent_t ev0 = nullptr, ev1 = nullptr;
    // host spill: track records moved off the device, one byte vector per
    // field of the track layout (the most recently spilled at the end)
    std::vector<char> spill_store[11];
    int64_t spill_n = 0;
    // tracks moved to host memory when the track slots could not hold the
    // next step (photons, charged): field arrays of over_n[r] records
    std::vector<char> over_store[2][11];
    int64_t over_n[2] = {0, 0};
    // pipelined schedule: queued interactions moved to host memory likewise
    std::vector<char> overq_store[13];
    int64_t overq_n = 0;
    // per-step records of emt_run_traced (null otherwise)
    emt_step_record* trace = nullptr;
    int32_t trace_cap = 0, trace_n = 0;

    template <typename T>
    T* at(size_t off) const { return reinterpret_cast<T*>(pool + off); }
    bool mixed() const { return plan.mixed; }
};

// tracks still to be stepped: in the track buffers, and (pipelined
// schedule) with an interaction queued for the next iteration
int64_t in_flight(const emt_ctx* c) { return c->live_g + c->live_c + c->live_q; }
// tracks waiting in host memory (host spill and slot overflow)
int64_t on_host(const emt_ctx* c) { return c->spill_n + c->over_n[0] + c->over_n[1] + c->overq_n; }

namespace {

emt_status fail(emt_ctx* c, emt_status s, const std::string& msg)
{
    if (c) c->err = msg;
    return s;
}

emt_status cuda_fail(emt_ctx* c, cudaError_t e, const char* where)
{
    if (c) {
        c->poisoned = true;
        c->err = std::string(where) + ": " + cudaGetErrorString(e);
    }
    return EMT_ERR_CUDA;
}

#define EMT_CUDA(c, expr)                                 \
    do {                                                  \
        cudaError_t e_ = (expr);                          \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, #expr); \
    } while (0)

template <typename R>
void fill_side(emt_ctx* c, Tracks<R>& q, const size_t* o)
{
    q.x = c->at<double>(o[0]);
    q.y = c->at<double>(o[1]);
    q.z = c->at<double>(o[2]);
    q.ux = c->at<R>(o[3]);
    q.uy = c->at<R>(o[4]);
    q.uz = c->at<R>(o[5]);
    q.T = c->at<R>(o[6]);
    q.uid = c->at<uint64_t>(o[7]);
    q.ev = c->at<uint32_t>(o[8]);
    q.step = c->at<uint32_t>(o[9]);
    q.tv = c->at<uint32_t>(o[10]);
}

template <typename R>
void fill_tracks(emt_ctx* c, Params<R>& p)
{
    if (c->plan.spill_on) fill_side(c, p.spill, c->plan.spill);
    for (int s = 0; s < 2; ++s) fill_side(c, p.q[s], c->plan.trk[s]);
}

template <typename R>
void fill_common(emt_ctx* c, Params<R>& p)
{
    const Plan& pl = c->plan;
    fill_tracks(c, p);
    auto fill_queue = [&](InterQueue<R>& q, const size_t* o) {
        q.x = c->at<double>(o[0]);
        q.y = c->at<double>(o[1]);
        q.z = c->at<double>(o[2]);
        q.ux = c->at<R>(o[3]);
        q.uy = c->at<R>(o[4]);
        q.uz = c->at<R>(o[5]);
        q.T = c->at<R>(o[6]);
        q.uid = c->at<uint64_t>(o[7]);
        q.dep = c->at<double>(o[8]);
        q.ev = c->at<uint32_t>(o[9]);
        q.step = c->at<uint32_t>(o[10]);
        q.tv = c->at<uint32_t>(o[11]);
        q.src = c->at<uint32_t>(o[12]);
    };
    if (pl.split) {
        fill_queue(p.iq, pl.iq);
        if (pl.pipelined) fill_queue(p.iq_alt, pl.iq_alt);
        p.skey = c->at<uint8_t>(pl.skey);
        p.sperm = c->at<uint32_t>(pl.sperm);
    }
    p.Q = pl.Q;
    p.cnt = c->at<Counters>(pl.cnt);
    p.status = c->at<int>(pl.status);
    p.total_steps = c->at<unsigned long long>(pl.total_steps);
    p.done_head = c->at<unsigned>(pl.done_head);
    p.hist = c->at<double>(pl.hist);
    p.hstride = pl.hstride;
    p.ledger = c->at<double>(pl.ledger);
    p.counts = c->at<unsigned long long>(pl.counts);
    p.live = c->at<int>(pl.live);
    p.event_id = c->at<uint64_t>(pl.event_id);
    p.done_ring = c->at<unsigned>(pl.done_ring);
    p.max_events = pl.max_events;
    p.seed = c->opt.seed;
    p.bk = c->at<double>(pl.bk);
    p.vacuum = c->at<int>(pl.vacuum);
    p.x0 = c->at<double>(pl.x0);
    p.ray_a = c->at<double>(pl.ray_a);
    p.zb = c->at<double>(pl.zb);
    p.lmat = c->at<int>(pl.lmat);
    p.lbin = c->at<int>(pl.lbin);
    p.step_bins = pl.step_bins;
    p.step_hist = pl.step_bins > 0 ? c->at<unsigned long long>(pl.step_hist) : nullptr;
    p.max_active = c->opt.max_active;
    p.select_policy = c->opt.select_policy;
    p.ehist = c->at<unsigned>(pl.ehist);
    p.spill_above = c->opt.spill_above;
    p.spill_cap = pl.spill_on ? pl.Q : 0;
    p.spill_ticket = c->at<int>(pl.spill_ticket);
}

void drop_graph(emt_ctx* c)
{
    if (c->graph) {
        cudaGraphExecDestroy(c->graph);
        c->graph = nullptr;
    }
}

// zero the score rows of the given slots and arm their submission token
__global__ void k_reset_slots(const uint32_t* slots, int n, double* hist, int hstride, double* ledger,
                              unsigned long long* counts, int* live, uint64_t* event_id, const uint64_t* ids)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t s = slots[i];
    for (int b = 0; b < hstride; ++b) hist[(size_t)s * hstride + b] = 0.0;
    ledger[3 * (size_t)s + 0] = 0.0;
    ledger[3 * (size_t)s + 1] = 0.0;
    ledger[3 * (size_t)s + 2] = 0.0;
    counts[2 * (size_t)s + 0] = 0;
    counts[2 * (size_t)s + 1] = 0;
    live[s] = 1;
    event_id[s] = ids[i];
}

// primaries must be contiguous per event; start[e] = first index, runs[e] =
// number of contiguous runs (must be <= 1); uid = rank within the event + 1
__global__ void k_runs(const int32_t* ev, int n, int n_events, uint32_t* start, uint32_t* runs, int* status)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int e = ev[i];
    if (e < 0 || e >= n_events) {
        atomicOr(status, 4);
        return;
    }
    if (i == 0 || ev[i - 1] != e) {
        atomicAdd(&runs[e], 1u);
        start[e] = (uint32_t)i;
    }
}

__global__ void k_uids(const int32_t* ev, int n, const uint32_t* start, const uint32_t* runs, uint32_t* uid,
                       int* status)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int e = ev[i];
    if (runs[e] != 1u) {
        atomicOr(status, 8);
        return;
    }
    uid[i] = (uint32_t)i - start[e] + 1u;
}

__global__ void k_release_tokens(const uint32_t* slots, int n, int* live, unsigned* done_ring, unsigned* done_head,
                                 int max_events)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t s = slots[i];
    int old = atomicAdd(&live[s], -1);
    if (old == 1) {
        unsigned k = atomicAdd(done_head, 1u);
        done_ring[k % (unsigned)max_events] = s;
    }
}

// per-event summary: {edep (sum of every column), escaped, killed, e_in,
// n_steps, n_tracks}
__global__ void k_gather(const uint32_t* slots, int n, const double* hist, int hstride, int n_bins,
                         const double* ledger, const unsigned long long* counts, double* out_hist,
                         double* out_summary)
{
    int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint32_t s = slots[i];
    const double* h = hist + (size_t)s * hstride;
    double edep = 0.0;
    for (int b = 0; b < n_bins; ++b) {
        if (out_hist) out_hist[(size_t)i * n_bins + b] = h[b];
        edep += h[b];
    }
    edep += h[n_bins];
    double* o = out_summary + (size_t)i * EMT_SUMMARY_LEN;
    o[0] = edep;
    o[1] = ledger[3 * (size_t)s + 0];
    o[2] = ledger[3 * (size_t)s + 1];
    o[3] = ledger[3 * (size_t)s + 2];
    o[4] = (double)counts[2 * (size_t)s + 0];
    o[5] = (double)counts[2 * (size_t)s + 1];
}

template <typename R>
Params<R>& params(emt_ctx* c);
template <>
Params<double>& params<double>(emt_ctx* c) { return c->pd; }
template <>
Params<float>& params<float>(emt_ctx* c) { return c->pf; }

emt_status sync_status(emt_ctx* c, const char* where)
{
    EMT_CUDA(c, cudaMemcpyAsync(c->h_status, c->pool + c->plan.status, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    EMT_CUDA(c, cudaStreamSynchronize(c->stream));
    if (*c->h_status & (int)kStatusQueueOverflow) {
        c->poisoned = true;
        return fail(c, EMT_ERR_CUDA, std::string(where) + ": track queue overflow (internal error)");
    }
    return EMT_OK;
}

// kernel launches of one step: the fused kernel; or the transport and
// interaction kernels, plus the two sorting launches of the charged tracks
// in a field (without track selection)
template <typename R>
int launches_per_step(const emt_ctx* c, const Params<R>& p)
{
    if (!c->plan.split) return 1;
    const int sort = (p.has_field && p.max_active <= 0) ? 2 : 0;
    return (c->plan.pipelined ? 1 : 2) + sort;
}

template <typename R>
emt_status run_loop(emt_ctx* c, int32_t max_iterations, emt_run_stats* st)
{
    Params<R>& p = params<R>(c);
    emt_run_stats s;
    std::memset(&s, 0, sizeof s);
    const Plan& pl = c->plan;
    c->head_fresh = false;
    const unsigned long long steps0 = c->steps_seen[0], def0 = c->steps_seen[1], held0 = c->steps_seen[2],
                             sub0 = c->steps_seen[3];
    unsigned long long last_steps = steps0;
    const int64_t live0 = in_flight(c);
    int64_t peak = live0;
    double kernel_ms = 0.0;
    unsigned long long deferred_prev = def0, held_prev = held0;
    Counters trace_cnt[3];
    // host spill: field sizes of a track record, and the refill rule (when
    // fewer than spill_above/2 tracks are on the device, move the most
    // recently spilled back, up to spill_above in total)
    const size_t rs = c->mixed() ? 4 : 8;
    const size_t fs[11] = {8, 8, 8, rs, rs, rs, rs, 8, 4, 4, 4};
    auto refill = [&]() -> emt_status {
        const int64_t N = c->live_g + c->live_c;
        if (c->spill_n == 0 || N >= c->opt.spill_above / 2) return EMT_OK;
        const int64_t n = std::min<int64_t>(c->spill_n, std::min<int64_t>(c->opt.spill_above - N, pl.Q - 2 - N));
        if (n <= 0) return EMT_OK;
        const int64_t first = c->spill_n - n;
        int64_t ng = 0;
        const uint32_t* tv = reinterpret_cast<const uint32_t*>(c->spill_store[10].data()) + first;
        for (int64_t k = 0; k < n; ++k) ng += (tv[k] & 0xFFu) == 0u;
        for (int f = 0; f < 11; ++f)
            EMT_CUDA(c, cudaMemcpyAsync(c->pool + pl.spill[f], c->spill_store[f].data() + fs[f] * first, fs[f] * n,
                                        cudaMemcpyHostToDevice, c->stream));
        EMT_CUDA(c, Launch<R>::unspill(p, (int)(c->it & 1), (int)(c->it % 3), (int)n, c->stream));
        EMT_CUDA(c, cudaStreamSynchronize(c->stream));
        for (int f = 0; f < 11; ++f) c->spill_store[f].resize(fs[f] * first);
        c->spill_n = first;
        c->live_g += ng;
        c->live_c += n - ng;
        return EMT_OK;
    };
    // after a step: move the tracks it spilled to host memory
    auto move_out = [&](int cin) -> emt_status {
        int spilled = 0;
        EMT_CUDA(c, cudaMemcpyAsync(&spilled, c->pool + pl.cnt + sizeof(Counters) * cin + offsetof(Counters, spilled),
                                    sizeof(int), cudaMemcpyDeviceToHost, c->stream));
        EMT_CUDA(c, cudaStreamSynchronize(c->stream));
        const int64_t n = std::min<int64_t>(spilled, pl.Q);
        if (n <= 0) return EMT_OK;
        for (int f = 0; f < 11; ++f) {
            c->spill_store[f].resize(fs[f] * (c->spill_n + n));
            EMT_CUDA(c, cudaMemcpyAsync(c->spill_store[f].data() + fs[f] * c->spill_n, c->pool + pl.spill[f],
                                        fs[f] * n, cudaMemcpyDeviceToHost, c->stream));
        }
        EMT_CUDA(c, cudaStreamSynchronize(c->stream));
        c->spill_n += n;
        s.spilled += n;
        s.peak_spilled = std::max<int64_t>(s.peak_spilled, c->spill_n);
        return EMT_OK;
    };
    // Slot overflow: every track's next step needs a second output slot and
    // none is free (a deterministic step repeats identically, so waiting
    // cannot help).  Half of each particle region, the tracks next to its
    // free end, moves to host memory with its state and step counter; they
    // come back when the device holds fewer than Q/4 tracks.  Results do not
    // change (each track's random stream is keyed on its own steps).
    // pipelined schedule: the queue that the next iteration samples, its
    // field sizes and its count (slot cs)
    const size_t qfs[13] = {8, 8, 8, rs, rs, rs, rs, 8, 8, 4, 4, 4, 4};
    auto pending_queue = [&](int64_t it) { return (it & 1) ? pl.iq : pl.iq_alt; };
    auto overflow_out = [&]() -> emt_status {
        const int side = (int)(c->it & 1), cs = (int)(c->it % 3);
        const int64_t nG = c->live_g, nC = c->live_c;
        const int64_t k[2] = {nG / 2, nC / 2};
        const int64_t kq = c->live_q / 2;
        if (k[0] + k[1] + kq == 0)
            return fail(c, EMT_ERR_CAPACITY, "no track could advance: slot_capacity is too small");
        if (kq > 0) {
            // the last kq records of the pending queue
            const size_t* qo = pending_queue(c->it);
            const int64_t nq = c->live_q;
            for (int f = 0; f < 13; ++f) {
                std::vector<char>& v = c->overq_store[f];
                const size_t old = v.size();
                v.resize(old + qfs[f] * kq);
                EMT_CUDA(c, cudaMemcpyAsync(v.data() + old, c->pool + qo[f] + qfs[f] * (nq - kq), qfs[f] * kq,
                                            cudaMemcpyDeviceToHost, c->stream));
            }
            const int nq2 = (int)(nq - kq);
            EMT_CUDA(c, cudaMemcpyAsync(c->pool + pl.cnt + sizeof(Counters) * cs + offsetof(Counters, n_int), &nq2,
                                        sizeof nq2, cudaMemcpyHostToDevice, c->stream));
            EMT_CUDA(c, cudaStreamSynchronize(c->stream));
            c->overq_n += kq;
            c->live_q = nq2;
            s.spilled += kq;
            s.peak_spilled = std::max<int64_t>(s.peak_spilled, on_host(c));
        }
        const int64_t first[2] = {nG - k[0], pl.Q - nC};  // photons: top of [0, nG); charged: bottom of [Q-nC, Q)
        for (int r = 0; r < 2; ++r) {
            if (k[r] == 0) continue;
            for (int f = 0; f < 11; ++f) {
                std::vector<char>& v = c->over_store[r][f];
                const size_t old = v.size();
                v.resize(old + fs[f] * k[r]);
                EMT_CUDA(c, cudaMemcpyAsync(v.data() + old, c->pool + pl.trk[side][f] + fs[f] * first[r],
                                            fs[f] * k[r], cudaMemcpyDeviceToHost, c->stream));
            }
            c->over_n[r] += k[r];
        }
        int n2[2] = {(int)(nG - k[0]), (int)(nC - k[1])};
        EMT_CUDA(c, cudaMemcpyAsync(c->pool + pl.cnt + sizeof(Counters) * cs + offsetof(Counters, n), n2, sizeof n2,
                                    cudaMemcpyHostToDevice, c->stream));
        EMT_CUDA(c, cudaStreamSynchronize(c->stream));
        c->live_g = n2[0];
        c->live_c = n2[1];
        s.spilled += k[0] + k[1];
        s.peak_spilled = std::max<int64_t>(s.peak_spilled, on_host(c));
        return EMT_OK;
    };
    auto overflow_in = [&]() -> emt_status {
        const int64_t N = in_flight(c);
        if (c->over_n[0] + c->over_n[1] + c->overq_n == 0 || N >= pl.Q / 4) return EMT_OK;
        int64_t budget = pl.Q / 2 - N;
        const int side = (int)(c->it & 1), cs = (int)(c->it % 3);
        if (c->overq_n > 0) {
            // queued interactions back to the end of the pending queue
            const int64_t k = std::min<int64_t>(c->overq_n, budget);
            const int64_t from = c->overq_n - k;
            const size_t* qo = pending_queue(c->it);
            for (int f = 0; f < 13; ++f)
                EMT_CUDA(c, cudaMemcpyAsync(c->pool + qo[f] + qfs[f] * c->live_q, c->overq_store[f].data() + qfs[f] * from,
                                            qfs[f] * k, cudaMemcpyHostToDevice, c->stream));
            const int nq2 = (int)(c->live_q + k);
            EMT_CUDA(c, cudaMemcpyAsync(c->pool + pl.cnt + sizeof(Counters) * cs + offsetof(Counters, n_int), &nq2,
                                        sizeof nq2, cudaMemcpyHostToDevice, c->stream));
            EMT_CUDA(c, cudaStreamSynchronize(c->stream));
            for (int f = 0; f < 13; ++f) c->overq_store[f].resize(qfs[f] * from);
            c->overq_n = from;
            c->live_q = nq2;
            budget -= k;
        }
        int64_t cnt2[2] = {c->live_g, c->live_c};
        for (int r = 0; r < 2 && budget > 0; ++r) {
            const int64_t k = std::min<int64_t>(c->over_n[r], budget);
            if (k <= 0) continue;
            const int64_t from = c->over_n[r] - k;  // the most recently moved out
            const int64_t to = r == 0 ? cnt2[0] : pl.Q - cnt2[1] - k;
            for (int f = 0; f < 11; ++f)
                EMT_CUDA(c, cudaMemcpyAsync(c->pool + pl.trk[side][f] + fs[f] * to,
                                            c->over_store[r][f].data() + fs[f] * from, fs[f] * k,
                                            cudaMemcpyHostToDevice, c->stream));
            EMT_CUDA(c, cudaStreamSynchronize(c->stream));
            for (int f = 0; f < 11; ++f) c->over_store[r][f].resize(fs[f] * from);
            c->over_n[r] = from;
            cnt2[r] += k;
            budget -= k;
        }
        int n2[2] = {(int)cnt2[0], (int)cnt2[1]};
        EMT_CUDA(c, cudaMemcpyAsync(c->pool + pl.cnt + sizeof(Counters) * cs + offsetof(Counters, n), n2, sizeof n2,
                                    cudaMemcpyHostToDevice, c->stream));
        EMT_CUDA(c, cudaStreamSynchronize(c->stream));
        c->live_g = n2[0];
        c->live_c = n2[1];
        return EMT_OK;
    };
    auto read_counts = [&]() -> emt_status {
        EMT_CUDA(c, cudaMemcpyAsync(c->h_cnt, c->pool + pl.cnt + sizeof(Counters) * (c->it % 3), sizeof(Counters),
                                    cudaMemcpyDeviceToHost, c->stream));
        EMT_CUDA(c, cudaStreamSynchronize(c->stream));
        float ms = 0.f;
        EMT_CUDA(c, cudaEventElapsedTime(&ms, c->ev0, c->ev1));
        kernel_ms += ms;
        const int64_t q = pl.pipelined ? (int64_t)c->h_cnt->n_int : 0;
        const bool same = c->live_g == c->h_cnt->n[0] && c->live_c == c->h_cnt->n[1] && c->live_q == q;
        c->live_g = c->h_cnt->n[0];
        c->live_c = c->h_cnt->n[1];
        c->live_q = q;
        peak = std::max<int64_t>(peak, in_flight(c));
        if (same && in_flight(c) > 0) {
            // unchanged population: make sure some track advanced
            EMT_CUDA(c, cudaMemcpyAsync(c->h_steps, c->pool + pl.total_steps, 16, cudaMemcpyDeviceToHost, c->stream));
            EMT_CUDA(c, cudaStreamSynchronize(c->stream));
            if (c->h_steps[0] == last_steps) {
                emt_status r = overflow_out();
                if (r != EMT_OK) return r;
            }
            last_steps = c->h_steps[0];
        }
        return EMT_OK;
    };
    auto one_plain = [&]() -> emt_status {
        if (pl.spill_on) {
            emt_status r0 = refill();
            if (r0 != EMT_OK) return r0;
        }
        {
            emt_status r0 = overflow_in();
            if (r0 != EMT_OK) return r0;
        }
        int side = (int)(c->it & 1), cin = (int)(c->it % 3), cout = (int)((c->it + 1) % 3),
            cclr = (int)((c->it + 2) % 3);
        int64_t chunks = (c->live_g + c->block - 1) / c->block + (c->live_c + c->block - 1) / c->block;
        int grid = (int)std::max<int64_t>(1, std::min<int64_t>(chunks, c->resident_blocks));
        EMT_CUDA(c, cudaEventRecord(c->ev0, c->stream));
        cudaError_t e =
            c->plan.pipelined
                ? Launch<R>::step_pipe(p, side, cin, cout, cclr, c->resident_p, c->resident_b, c->block, c->stream)
            : c->plan.split
                ? Launch<R>::step_split(p, side, cin, cout, cclr,
                                        (int)std::max<int64_t>(1, std::min<int64_t>(chunks, c->resident_a)),
                                        c->resident_b, c->block, c->stream)
                : Launch<R>::step(p, side, cin, cout, cclr, grid, c->block, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "step kernel launch");
        EMT_CUDA(c, cudaEventRecord(c->ev1, c->stream));
        s.kernel_launches += launches_per_step(c, p);
        c->it += 1;
        s.iterations += 1;
        const int64_t g0 = c->live_g, c0 = c->live_c;
        const double ms0 = kernel_ms;
        emt_status r = read_counts();
        if (r == EMT_OK && pl.spill_on) r = move_out(cin);
        if (r != EMT_OK || !c->trace || c->trace_n >= c->trace_cap) return r;
        // per-step record: the input counters of this step hold its
        // interaction count; the step counters give the deferred copies
        EMT_CUDA(c, cudaMemcpyAsync(trace_cnt, c->pool + pl.cnt, sizeof trace_cnt, cudaMemcpyDeviceToHost, c->stream));
        EMT_CUDA(c, cudaMemcpyAsync(c->h_steps, c->pool + pl.total_steps, 24, cudaMemcpyDeviceToHost, c->stream));
        EMT_CUDA(c, cudaStreamSynchronize(c->stream));
        emt_step_record& rec = c->trace[c->trace_n++];
        rec.photons = g0;
        rec.charged = c0;
        rec.interacting = c->plan.split ? (int64_t)trace_cnt[cin].n_int : -1;
        rec.deferred = (int64_t)(c->h_steps[1] - deferred_prev);
        deferred_prev = c->h_steps[1];
        rec.held = (int64_t)(c->h_steps[2] - held_prev);
        held_prev = c->h_steps[2];
        rec.ms = kernel_ms - ms0;
        return EMT_OK;
    };
    int64_t done_it = 0;
    auto budget_left = [&]() { return max_iterations <= 0 || done_it < max_iterations; };
    if (c->opt.loop_mode == EMT_LOOP_PLAIN || c->trace || pl.spill_on) {
        while ((in_flight(c) > 0 || on_host(c) > 0) && budget_left()) {
            emt_status r = one_plain();
            if (r != EMT_OK) return r;
            ++done_it;
        }
    } else if (c->opt.loop_mode == EMT_LOOP_PERSISTENT) {
        // up to graph_steps steps per cooperative launch; the launch ends
        // early when no track is left and reports how many steps it ran
        GridSync* gs = c->at<GridSync>(pl.gsync);
        while ((in_flight(c) > 0 || on_host(c) > 0) && budget_left()) {
            const int k = max_iterations > 0 ? (int)std::min<int64_t>(c->opt.graph_steps, max_iterations - done_it)
                                             : c->opt.graph_steps;
            {
                emt_status r0 = overflow_in();
                if (r0 != EMT_OK) return r0;
            }
            EMT_CUDA(c, cudaMemsetAsync(gs, 0, sizeof(GridSync), c->stream));
            EMT_CUDA(c, cudaEventRecord(c->ev0, c->stream));
            cudaError_t e = Launch<R>::persist(p, c->it, k, gs, c->wait_cycles, c->persist_grid, c->block, c->stream);
            if (e != cudaSuccess) return cuda_fail(c, e, "persistent step loop launch");
            EMT_CUDA(c, cudaEventRecord(c->ev1, c->stream));
            GridSync h_gs;
            EMT_CUDA(c, cudaMemcpyAsync(&h_gs, gs, sizeof h_gs, cudaMemcpyDeviceToHost, c->stream));
            EMT_CUDA(c, cudaMemcpyAsync(c->h_status, c->pool + pl.status, sizeof(int), cudaMemcpyDeviceToHost,
                                        c->stream));
            EMT_CUDA(c, cudaStreamSynchronize(c->stream));
            if (*c->h_status & kStatusTimeout) {
                // the steps of this launch are incomplete: the context's
                // track state is no longer consistent
                c->poisoned = true;
                return fail(c, EMT_ERR_TIMEOUT, "persistent step loop: a grid barrier wait gave up");
            }
            s.kernel_launches += 1;
            c->it += h_gs.iters;
            s.iterations += h_gs.iters;
            done_it += h_gs.iters;
            emt_status r = read_counts();
            if (r != EMT_OK) return r;
        }
    } else {
        const int K = c->opt.graph_steps;
        while ((in_flight(c) > 0 || on_host(c) > 0) && budget_left()) {
            if (c->it % 6 != 0 || (max_iterations > 0 && max_iterations - done_it < K)) {
                emt_status r = one_plain();
                if (r != EMT_OK) return r;
                ++done_it;
                continue;
            }
            if (!c->graph) {
                cudaGraph_t g;
                EMT_CUDA(c, cudaStreamBeginCapture(c->stream, cudaStreamCaptureModeThreadLocal));
                for (int k = 0; k < K; ++k) {
                    int side = k & 1, cin = k % 3, cout = (k + 1) % 3, cclr = (k + 2) % 3;
                    cudaError_t e = c->plan.pipelined
                                        ? Launch<R>::step_pipe(p, side, cin, cout, cclr, c->resident_p, c->resident_b,
                                                               c->block, c->stream)
                                    : c->plan.split ? Launch<R>::step_split(p, side, cin, cout, cclr, c->resident_a,
                                                                          c->resident_b, c->block, c->stream)
                                                  : Launch<R>::step(p, side, cin, cout, cclr, c->resident_blocks,
                                                                    c->block, c->stream);
                    if (e != cudaSuccess) {
                        cudaStreamEndCapture(c->stream, &g);
                        return cuda_fail(c, e, "graph capture");
                    }
                }
                EMT_CUDA(c, cudaStreamEndCapture(c->stream, &g));
                EMT_CUDA(c, cudaGraphInstantiate(&c->graph, g, 0));
                cudaGraphDestroy(g);
            }
            {
                emt_status r0 = overflow_in();
                if (r0 != EMT_OK) return r0;
            }
            EMT_CUDA(c, cudaEventRecord(c->ev0, c->stream));
            EMT_CUDA(c, cudaGraphLaunch(c->graph, c->stream));
            EMT_CUDA(c, cudaEventRecord(c->ev1, c->stream));
            s.kernel_launches += K * launches_per_step(c, p);
            c->it += K;
            s.iterations += K;
            done_it += K;
            emt_status r = read_counts();
            if (r != EMT_OK) return r;
        }
    }
    // status word, step counters and finished-event head in one copy
    const size_t misc = pl.done_head + sizeof(unsigned) - pl.status;
    EMT_CUDA(c, cudaMemcpyAsync(c->h_misc, c->pool + pl.status, misc, cudaMemcpyDeviceToHost, c->stream));
    EMT_CUDA(c, cudaStreamSynchronize(c->stream));
    const int status = *reinterpret_cast<const int*>(c->h_misc);
    const unsigned long long* steps = reinterpret_cast<const unsigned long long*>(c->h_misc + (pl.total_steps - pl.status));
    c->steps_seen[0] = steps[0];
    c->steps_seen[1] = steps[1];
    c->steps_seen[2] = steps[2];
    c->steps_seen[3] = steps[3];
    c->head_cached = *reinterpret_cast<const unsigned*>(c->h_misc + (pl.done_head - pl.status));
    c->head_fresh = true;
    if (status & (int)kStatusQueueOverflow) {
        c->poisoned = true;
        return fail(c, EMT_ERR_CUDA, "emt_run: track queue overflow (internal error)");
    }
    s.track_steps = (int64_t)(c->steps_seen[0] - steps0);
    s.deferred = (int64_t)(c->steps_seen[1] - def0);
    s.held = (int64_t)(c->steps_seen[2] - held0);
    s.rk4_substeps = (int64_t)(c->steps_seen[3] - sub0);
    s.peak_tracks = peak;
    s.live_tracks = in_flight(c) + on_host(c);
    s.kernel_ms = kernel_ms;
    // every launch reads its inputs and writes its outputs once; the
    // outputs of one launch are the inputs of the next
    const int64_t n_in = s.track_steps + s.deferred + s.held;
    const int64_t slot_bytes = c->mixed() ? 60 : 76;
    s.state_bytes = (2 * n_in - live0 + s.live_tracks) * slot_bytes;
    if (st) *st = s;
    return EMT_OK;
}

emt_status check_ready(emt_ctx* c)
{
    if (!c) return EMT_ERR_INVALID_ARG;
    if (c->poisoned) return fail(c, EMT_ERR_CUDA, "context unusable after an earlier CUDA error");
    if (!c->have_materials || !c->have_geometry)
        return fail(c, EMT_ERR_BAD_STATE, "load materials and geometry first");
    if (cudaSetDevice(c->opt.device) != cudaSuccess) return fail(c, EMT_ERR_CUDA, "cudaSetDevice");
    return EMT_OK;
}

// read the finished-event ring into slot states
emt_status drain_done(emt_ctx* c)
{
    const Plan& pl = c->plan;
    unsigned head = c->head_cached;
    if (!c->head_fresh) {
        EMT_CUDA(c, cudaMemcpyAsync(c->h_done, c->pool + pl.done_head, sizeof(unsigned), cudaMemcpyDeviceToHost,
                                    c->stream));
        EMT_CUDA(c, cudaStreamSynchronize(c->stream));
        head = *c->h_done;
        c->head_cached = head;
    }
    if (head == c->done_seen) return EMT_OK;
    unsigned n = head - c->done_seen;
    if (n > (unsigned)pl.max_events) return fail(c, EMT_ERR_CUDA, "finished-event ring overrun");
    std::vector<unsigned> ring(pl.max_events);
    EMT_CUDA(c, cudaMemcpyAsync(ring.data(), c->pool + pl.done_ring, sizeof(unsigned) * pl.max_events,
                                cudaMemcpyDeviceToHost, c->stream));
    EMT_CUDA(c, cudaStreamSynchronize(c->stream));
    for (unsigned k = c->done_seen; k != head; ++k) {
        unsigned s = ring[k % (unsigned)pl.max_events];
        if (s < c->slot_state.size() && c->slot_state[s] == 1) c->slot_state[s] = 2;
    }
    c->done_seen = head;
    return EMT_OK;
}

void release_slot(emt_ctx* c, int s)
{
    c->id_to_slot.erase(c->slot_id[s]);
    c->slot_state[s] = 0;
    c->free_slots.push_back(s);
}

}  // namespace

extern "C" {

void emt_default_options(emt_options* o)
{
    if (!o) return;
    std::memset(o, 0, sizeof *o);
    o->device = 0;
    o->precision = EMT_PRECISION_FP64;
    o->slot_capacity = (int64_t)1 << 22;
    o->max_events = 10000;
    o->max_bins = 128;
    o->block_size = 0;
    o->loop_mode = EMT_LOOP_PLAIN;
    o->graph_steps = 12;
    o->schedule = EMT_SCHEDULE_FUSED;
    o->seed = 1;
}

size_t emt_pool_bytes(const emt_options* o)
{
    if (!o) return 0;
    std::string why;
    if (!valid_options(*o, why)) return 0;
    return make_plan(*o).total;
}

emt_status emt_create(const emt_options* o, emt_ctx** out)
{
    if (!o || !out) return EMT_ERR_INVALID_ARG;
    *out = nullptr;
    std::string why;
    if (!valid_options(*o, why)) return EMT_ERR_INVALID_ARG;
    emt_ctx* c = new (std::nothrow) emt_ctx();
    if (!c) return EMT_ERR_HOST_OOM;
    c->opt = *o;
    c->plan = make_plan(*o);
    auto bail = [&](emt_status s) {
        emt_destroy(c);
        return s;
    };
    if (cudaSetDevice(o->device) != cudaSuccess) return bail(EMT_ERR_CUDA);
    if (o->cuda_stream) {
        c->stream = (cudaStream_t)o->cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking) != cudaSuccess) return bail(EMT_ERR_CUDA);
        c->own_stream = true;
    }
    if (o->device_pool) {
        if (o->pool_bytes < c->plan.total || ((uintptr_t)o->device_pool % kAlign) != 0) return bail(EMT_ERR_INVALID_ARG);
        c->pool = (char*)o->device_pool;
    } else {
        if (cudaMalloc((void**)&c->pool, c->plan.total) != cudaSuccess) return bail(EMT_ERR_CUDA);
        c->own_pool = true;
    }
    if (cudaMallocHost((void**)&c->h_cnt, sizeof(Counters)) != cudaSuccess ||
        cudaMallocHost((void**)&c->h_status, sizeof(int)) != cudaSuccess ||
        cudaMallocHost((void**)&c->h_steps, 4 * sizeof(unsigned long long)) != cudaSuccess ||
        cudaMallocHost((void**)&c->h_done, sizeof(unsigned)) != cudaSuccess ||
        cudaMallocHost((void**)&c->h_misc, make_plan(*o).done_head + sizeof(unsigned) - make_plan(*o).status) !=
            cudaSuccess)
        return bail(EMT_ERR_CUDA);
    if (cudaEventCreate(&c->ev0) != cudaSuccess || cudaEventCreate(&c->ev1) != cudaSuccess) return bail(EMT_ERR_CUDA);
    const Plan& pl = c->plan;
    // counters, status and score metadata start at zero
    if (cudaMemsetAsync(c->pool + pl.cnt, 0, pl.hist - pl.cnt, c->stream) != cudaSuccess) return bail(EMT_ERR_CUDA);
    if (cudaMemsetAsync(c->pool + pl.live, 0, pl.grid - pl.live, c->stream) != cudaSuccess) return bail(EMT_ERR_CUDA);
    if (pl.step_bins > 0 &&
        cudaMemsetAsync(c->pool + pl.step_hist, 0, (size_t)3 * pl.step_bins * sizeof(unsigned long long), c->stream) !=
            cudaSuccess)
        return bail(EMT_ERR_CUDA);
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return bail(EMT_ERR_CUDA);
    fill_common(c, c->pd);
    fill_common(c, c->pf);
    c->block = o->block_size ? o->block_size : 256;
    int dev_sms = 0;
    cudaDeviceGetAttribute(&dev_sms, cudaDevAttrMultiProcessorCount, o->device);
    int per_sm = c->mixed() ? Launch<float>::max_blocks_per_sm(c->block) : Launch<double>::max_blocks_per_sm(c->block);
    c->resident_blocks = std::max(1, dev_sms * per_sm);
    if (c->plan.split) {
        auto blocks = [&](int which) {
            return c->mixed() ? Launch<float>::max_blocks_split(c->block, which)
                              : Launch<double>::max_blocks_split(c->block, which);
        };
        c->resident_a = std::max(1, dev_sms * blocks(0));
        c->resident_b = std::max(1, dev_sms * blocks(1));
        if (c->plan.pipelined)
            c->resident_p = std::max(1, dev_sms * (c->mixed() ? Launch<float>::max_blocks_pipe(c->block)
                                                              : Launch<double>::max_blocks_pipe(c->block)));
    }
    if (o->loop_mode == EMT_LOOP_PERSISTENT) {
        int coop = 0, clock_khz = 0;
        cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, o->device);
        cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, o->device);
        const int per = c->mixed() ? Launch<float>::persist_blocks_per_sm(c->block)
                                   : Launch<double>::persist_blocks_per_sm(c->block);
        if (!coop || per < 1 || clock_khz < 1) {
            why = "the device cannot run the persistent step loop (cooperative launch)";
            return bail(EMT_ERR_INVALID_ARG);
        }
        c->persist_grid = dev_sms * per;
        c->wait_cycles = (long long)(kPersistWaitMs * (double)clock_khz);
    }
    c->slot_id.assign(pl.max_events, 0);
    c->slot_state.assign(pl.max_events, 0);
    c->free_slots.reserve(pl.max_events);
    for (int s = pl.max_events - 1; s >= 0; --s) c->free_slots.push_back(s);
    *out = c;
    return EMT_OK;
}

void emt_destroy(emt_ctx* c)
{
    if (!c) return;
    cudaSetDevice(c->opt.device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    drop_graph(c);
    if (c->own_pool && c->pool) cudaFree(c->pool);
    if (c->h_cnt) cudaFreeHost(c->h_cnt);
    if (c->h_status) cudaFreeHost(c->h_status);
    if (c->h_steps) cudaFreeHost(c->h_steps);
    if (c->h_done) cudaFreeHost(c->h_done);
    if (c->h_misc) cudaFreeHost(c->h_misc);
    if (c->ev0) cudaEventDestroy(c->ev0);
    if (c->ev1) cudaEventDestroy(c->ev1);
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

const char* emt_last_error(const emt_ctx* c) { return c ? c->err.c_str() : "null context"; }

emt_status emt_load_materials(emt_ctx* c, const emt_material* mats, int32_t n, const emt_physics* ph)
{
    if (!c || !mats || !ph) return fail(c, EMT_ERR_INVALID_ARG, "null argument");
    if (c->poisoned) return fail(c, EMT_ERR_CUDA, "context unusable");
    if (n < 1 || n > kMaxMat) return fail(c, EMT_ERR_INVALID_ARG, "material count out of [1, 16]");
    if (!(ph->grid_lo_MeV > 0.0) || !(ph->grid_hi_MeV > ph->grid_lo_MeV) || ph->bins_per_decade < 1)
        return fail(c, EMT_ERR_INVALID_ARG, "energy grid");
    double nint = ph->bins_per_decade * std::log10(ph->grid_hi_MeV / ph->grid_lo_MeV);
    int n_grid = (int)std::floor(nint + 0.5) + 1;
    if (n_grid < 2 || n_grid > kMaxGrid) return fail(c, EMT_ERR_INVALID_ARG, "grid must have 2..129 nodes");
    for (int k = 0; k < 3; ++k)
        if (!(ph->cut_MeV[k] > 0.0)) return fail(c, EMT_ERR_INVALID_ARG, "cuts must be positive");
    if (!(ph->step_frac > 0.0) || !(ph->final_range_cm > 0.0)) return fail(c, EMT_ERR_INVALID_ARG, "step limits");
    std::vector<MaterialDev> md(n);
    std::vector<double> bk(n);
    std::vector<int> vac(n);
    for (int i = 0; i < n; ++i) {
        const emt_material& m = mats[i];
        bool vacuum = !(m.rho_g_cm3 > 0.0);
        if (!vacuum && (!(m.Z >= 1.0) || !(m.A_g_mol > 0.0) || !(m.I_eV > 0.0) || !(m.bk_MeV >= 0.0)))
            return fail(c, EMT_ERR_INVALID_ARG, "material parameters");
        md[i] = {m.Z, m.A_g_mol, vacuum ? 0.0 : m.rho_g_cm3, m.I_eV, m.bk_MeV};
        bk[i] = m.bk_MeV;
        vac[i] = vacuum ? 1 : 0;
    }
    if (cudaSetDevice(c->opt.device) != cudaSuccess) return fail(c, EMT_ERR_CUDA, "cudaSetDevice");
    const Plan& pl = c->plan;
    EMT_CUDA(c, cudaMemcpyAsync(c->pool + pl.mats, md.data(), sizeof(MaterialDev) * n, cudaMemcpyHostToDevice, c->stream));
    EMT_CUDA(c, cudaMemcpyAsync(c->pool + pl.bk, bk.data(), sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
    EMT_CUDA(c, cudaMemcpyAsync(c->pool + pl.vacuum, vac.data(), sizeof(int) * n, cudaMemcpyHostToDevice, c->stream));
    TableBuild b;
    b.mats = c->at<MaterialDev>(pl.mats);
    b.n_mat = n;
    b.n_grid = n_grid;
    b.bpd = ph->bins_per_decade;
    b.e_lo = ph->grid_lo_MeV;
    for (int k = 0; k < 3; ++k) b.cut[k] = ph->cut_MeV[k];
    b.mask = ph->process_mask;
    b.x0 = c->at<double>(pl.x0);
    b.ray_a = c->at<double>(pl.ray_a);
    b.grid = c->at<double>(pl.grid);
    b.tab = c->at<double>(pl.tab);
    b.dedx = c->at<double>(pl.dedx);
    b.tabf = c->mixed() ? c->at<float>(pl.tabf) : nullptr;
    b.gridf = c->mixed() ? c->at<float>(pl.gridf) : nullptr;
    b.igrid = c->at<double>(pl.igrid);
    b.irs = c->at<double>(pl.irs);
    b.igridf = c->mixed() ? c->at<float>(pl.igridf) : nullptr;
    b.irsf = c->mixed() ? c->at<float>(pl.irsf) : nullptr;
    b.dgrid = c->at<double>(pl.dgrid);
    b.dtab = c->at<double>(pl.dtab);
    b.dgridf = c->mixed() ? c->at<float>(pl.dgridf) : nullptr;
    b.dtabf = c->mixed() ? c->at<float>(pl.dtabf) : nullptr;
    EMT_CUDA(c, build_tables(b, c->at<double>(pl.scratch), c->stream));
    EMT_CUDA(c, cudaStreamSynchronize(c->stream));
    c->n_mat = n;
    c->n_grid = n_grid;
    float l10 = (float)std::log10(ph->grid_lo_MeV);
    for (int k = 0; k < 3; ++k) {
        c->pd.cut[k] = ph->cut_MeV[k];
        c->pf.cut[k] = ph->cut_MeV[k];
        c->pd.cutf[k] = c->pf.cutf[k] = (float)ph->cut_MeV[k];
    }
    c->pd.grid = b.grid;
    c->pd.tab = b.tab;
    c->pf.grid = c->at<float>(pl.gridf);
    c->pf.tab = c->at<float>(pl.tabf);
    c->pd.igrid = b.igrid;
    c->pd.irs = b.irs;
    c->pf.igrid = c->at<float>(pl.igridf);
    c->pf.irs = c->at<float>(pl.irsf);
    c->pd.dgrid = b.dgrid;
    c->pd.dtab = b.dtab;
    c->pf.dgrid = c->at<float>(pl.dgridf);
    c->pf.dtab = c->at<float>(pl.dtabf);
    c->pd.n_grid = c->pf.n_grid = n_grid;
    c->pd.bpd = c->pf.bpd = ph->bins_per_decade;
    c->pd.log10_lo = c->pf.log10_lo = l10;
    c->pd.step_frac = c->pf.step_frac = ph->step_frac;
    c->pd.mask = c->pf.mask = ph->process_mask;
    c->pd.final_range = c->pf.final_range = ph->final_range_cm;
    c->pd.step_fracf = c->pf.step_fracf = (float)ph->step_frac;
    c->pd.final_rangef = c->pf.final_rangef = (float)ph->final_range_cm;
    drop_graph(c);
    c->have_materials = true;
    return EMT_OK;
}

emt_status emt_load_geometry(emt_ctx* c, const emt_layer* layers, int32_t n, const emt_world* w)
{
    if (!c || !layers || !w) return fail(c, EMT_ERR_INVALID_ARG, "null argument");
    if (c->poisoned) return fail(c, EMT_ERR_CUDA, "context unusable");
    if (!c->have_materials) return fail(c, EMT_ERR_BAD_STATE, "load materials first");
    if (n < 1 || n > kMaxLayers) return fail(c, EMT_ERR_INVALID_ARG, "layer count out of [1, 4096]");
    std::vector<double> zb(n + 1);
    std::vector<int> lm(n), lb(n);
    if (const char* why = check_geometry(layers, n, w, c->n_mat, c->opt.max_bins, zb.data(), lm.data(), lb.data()))
        return fail(c, EMT_ERR_INVALID_ARG, why);
    if (cudaSetDevice(c->opt.device) != cudaSuccess) return fail(c, EMT_ERR_CUDA, "cudaSetDevice");
    const Plan& pl = c->plan;
    EMT_CUDA(c, cudaMemcpyAsync(c->pool + pl.zb, zb.data(), sizeof(double) * (n + 1), cudaMemcpyHostToDevice, c->stream));
    EMT_CUDA(c, cudaMemcpyAsync(c->pool + pl.lmat, lm.data(), sizeof(int) * n, cudaMemcpyHostToDevice, c->stream));
    EMT_CUDA(c, cudaMemcpyAsync(c->pool + pl.lbin, lb.data(), sizeof(int) * n, cudaMemcpyHostToDevice, c->stream));
    EMT_CUDA(c, cudaStreamSynchronize(c->stream));
    set_geometry(c->pd, n, w);
    set_geometry(c->pf, n, w);
    c->n_layers = n;
    c->n_bins = w->n_bins;
    drop_graph(c);
    c->have_geometry = true;
    return EMT_OK;
}

}  // extern "C"

template <typename R>
static emt_status submit_impl(emt_ctx* c, int32_t n_events, const uint64_t* ids, const emt_primaries* pr, int32_t where)
{
    const Plan& pl = c->plan;
    const int n = pr->n;
    if ((int64_t)n > pl.max_prim) return fail(c, EMT_ERR_CAPACITY, "too many primaries in one submit");
    if ((int64_t)c->free_slots.size() < n_events) return fail(c, EMT_ERR_CAPACITY, "no free event slots");
    if (in_flight(c) + n > pl.Q - 2) return fail(c, EMT_ERR_CAPACITY, "no free track slots");
    for (int e = 0; e < n_events; ++e)
        if (c->id_to_slot.count(ids[e])) return fail(c, EMT_ERR_INVALID_ARG, "event id already in flight");
    {
        std::unordered_map<uint64_t, int> seen;
        for (int e = 0; e < n_events; ++e)
            if (!seen.emplace(ids[e], e).second) return fail(c, EMT_ERR_INVALID_ARG, "duplicate event id");
    }
    if (where == EMT_HOST) {
        for (int i = 0; i < n; ++i) {
            if (pr->event[i] < 0 || pr->event[i] >= n_events) return fail(c, EMT_ERR_INVALID_ARG, "event index");
            if (pr->type[i] < 0 || pr->type[i] > 2) return fail(c, EMT_ERR_INVALID_ARG, "particle type");
            if (!(pr->T_MeV[i] > 0.0) || !std::isfinite(pr->T_MeV[i])) return fail(c, EMT_ERR_INVALID_ARG, "energy");
            const double* d = pr->dir + 3 * (size_t)i;
            double nn = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
            if (!(std::fabs(nn - 1.0) < 1e-6)) return fail(c, EMT_ERR_INVALID_ARG, "direction not a unit vector");
        }
    }
    // slots
    std::vector<uint32_t> slots(n_events);
    for (int e = 0; e < n_events; ++e) {
        slots[e] = (uint32_t)c->free_slots.back();
        c->free_slots.pop_back();
    }
    auto undo = [&]() {
        for (int e = n_events - 1; e >= 0; --e) c->free_slots.push_back((int)slots[e]);
    };
    const int32_t *ev = pr->event, *ty = pr->type;
    const double *T = pr->T_MeV, *pos = pr->pos_cm, *dir = pr->dir;
    cudaStream_t st = c->stream;
    auto cp = [&](size_t off, const void* src, size_t bytes) {
        return cudaMemcpyAsync(c->pool + off, src, bytes, where == EMT_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice, st);
    };
    if (n > 0) {
        cudaError_t e1 = cp(pl.st_ev, ev, 4 * (size_t)n);
        if (e1 == cudaSuccess) e1 = cp(pl.st_type, ty, 4 * (size_t)n);
        if (e1 == cudaSuccess) e1 = cp(pl.st_T, T, 8 * (size_t)n);
        if (e1 == cudaSuccess) e1 = cp(pl.st_pos, pos, 24 * (size_t)n);
        if (e1 == cudaSuccess) e1 = cp(pl.st_dir, dir, 24 * (size_t)n);
        if (e1 != cudaSuccess) {
            undo();
            return cuda_fail(c, e1, "copy primaries");
        }
    }
    EMT_CUDA(c, cudaMemcpyAsync(c->pool + pl.st_slot, slots.data(), 4 * (size_t)n_events, cudaMemcpyHostToDevice, st));
    EMT_CUDA(c, cudaMemcpyAsync(c->pool + pl.st_ids, ids, 8 * (size_t)n_events, cudaMemcpyHostToDevice, st));
    EMT_CUDA(c, cudaMemsetAsync(c->pool + pl.st_runs, 0, 4 * (size_t)n_events, st));
    EMT_CUDA(c, cudaMemsetAsync(c->pool + pl.status, 0, sizeof(int), st));
    if (n > 0) {
        k_runs<<<(n + 255) / 256, 256, 0, st>>>(c->at<int32_t>(pl.st_ev), n, n_events, c->at<uint32_t>(pl.st_start),
                                                c->at<uint32_t>(pl.st_runs), c->at<int>(pl.status));
        k_uids<<<(n + 255) / 256, 256, 0, st>>>(c->at<int32_t>(pl.st_ev), n, c->at<uint32_t>(pl.st_start),
                                                c->at<uint32_t>(pl.st_runs), c->at<uint32_t>(pl.st_uid),
                                                c->at<int>(pl.status));
    }
    EMT_CUDA(c, cudaGetLastError());
    EMT_CUDA(c, cudaMemcpyAsync(c->h_status, c->pool + pl.status, sizeof(int), cudaMemcpyDeviceToHost, st));
    EMT_CUDA(c, cudaStreamSynchronize(st));
    if (*c->h_status != 0) {
        undo();
        return fail(c, EMT_ERR_INVALID_ARG,
                    (*c->h_status & 4) ? "event index out of range" : "primaries of an event must be contiguous");
    }
    k_reset_slots<<<(n_events + 127) / 128, 128, 0, st>>>(c->at<uint32_t>(pl.st_slot), n_events, c->at<double>(pl.hist),
                                                          pl.hstride, c->at<double>(pl.ledger),
                                                          c->at<unsigned long long>(pl.counts), c->at<int>(pl.live),
                                                          c->at<uint64_t>(pl.event_id), c->at<uint64_t>(pl.st_ids));
    EMT_CUDA(c, cudaGetLastError());
    Params<R>& p = params<R>(c);
    int side = (int)(c->it & 1), cs = (int)(c->it % 3);
    c->head_fresh = false;  // admission may finish events (token release)
    EMT_CUDA(c, Launch<R>::admit(p, side, cs, n, c->at<int32_t>(pl.st_ev), c->at<int32_t>(pl.st_type),
                                 c->at<double>(pl.st_T), c->at<double>(pl.st_pos), c->at<double>(pl.st_dir),
                                 c->at<uint32_t>(pl.st_slot), c->at<uint32_t>(pl.st_uid), st));
    k_release_tokens<<<(n_events + 127) / 128, 128, 0, st>>>(c->at<uint32_t>(pl.st_slot), n_events, c->at<int>(pl.live),
                                                             c->at<unsigned>(pl.done_ring), c->at<unsigned>(pl.done_head),
                                                             pl.max_events);
    EMT_CUDA(c, cudaGetLastError());
    EMT_CUDA(c, cudaMemcpyAsync(c->h_cnt, c->pool + pl.cnt + sizeof(Counters) * cs, sizeof(Counters),
                                cudaMemcpyDeviceToHost, st));
    EMT_CUDA(c, cudaMemcpyAsync(c->h_status, c->pool + pl.status, sizeof(int), cudaMemcpyDeviceToHost, st));
    EMT_CUDA(c, cudaStreamSynchronize(st));
    if (*c->h_status & kStatusBadTrack) {
        c->poisoned = true;
        return fail(c, EMT_ERR_INVALID_ARG, "invalid particle type in device primaries (context reset needed)");
    }
    if (*c->h_status & kStatusQueueOverflow) {
        c->poisoned = true;
        return fail(c, EMT_ERR_CUDA, "track queue overflow at admission");
    }
    c->live_g = c->h_cnt->n[0];
    c->live_c = c->h_cnt->n[1];
    for (int e = 0; e < n_events; ++e) {
        int s = (int)slots[e];
        c->slot_id[s] = ids[e];
        c->slot_state[s] = 1;
        c->id_to_slot[ids[e]] = s;
        c->order.push_back(s);
    }
    return EMT_OK;
}

extern "C" {

emt_status emt_submit(emt_ctx* c, int32_t n_events, const uint64_t* ids, const emt_primaries* pr, int32_t where)
{
    emt_status r = check_ready(c);
    if (r != EMT_OK) return r;
    if (n_events < 1 || !ids || !pr || pr->n < 0) return fail(c, EMT_ERR_INVALID_ARG, "bad submit arguments");
    if (pr->n > 0 && (!pr->event || !pr->type || !pr->T_MeV || !pr->pos_cm || !pr->dir))
        return fail(c, EMT_ERR_INVALID_ARG, "null primary array");
    if (where != EMT_HOST && where != EMT_DEVICE) return fail(c, EMT_ERR_INVALID_ARG, "where");
    return c->mixed() ? submit_impl<float>(c, n_events, ids, pr, where) : submit_impl<double>(c, n_events, ids, pr, where);
}

emt_status emt_run(emt_ctx* c, int32_t max_iterations, emt_run_stats* st)
{
    emt_status r = check_ready(c);
    if (r != EMT_OK) return r;
    r = c->mixed() ? run_loop<float>(c, max_iterations, st) : run_loop<double>(c, max_iterations, st);
    if (r != EMT_OK) return r;
    return drain_done(c);
}

emt_status emt_run_traced(emt_ctx* c, int32_t max_iterations, emt_run_stats* st, emt_step_record* rec, int32_t cap,
                          int32_t* n_rec)
{
    emt_status r = check_ready(c);
    if (r != EMT_OK) return r;
    if (!n_rec || cap < 0 || (cap > 0 && !rec)) return fail(c, EMT_ERR_INVALID_ARG, "trace buffer");
    c->trace = rec;
    c->trace_cap = cap;
    c->trace_n = 0;
    r = c->mixed() ? run_loop<float>(c, max_iterations, st) : run_loop<double>(c, max_iterations, st);
    *n_rec = c->trace_n;
    c->trace = nullptr;
    c->trace_cap = c->trace_n = 0;
    if (r != EMT_OK) return r;
    return drain_done(c);
}

emt_status emt_read_step_hist(emt_ctx* c, uint64_t* out, int32_t bins, int32_t reset)
{
    if (!c) return EMT_ERR_INVALID_ARG;
    if (c->poisoned) return fail(c, EMT_ERR_CUDA, "context unusable after an earlier CUDA error");
    if (c->plan.step_bins <= 0) return fail(c, EMT_ERR_BAD_STATE, "the steps-per-track histogram is off");
    if (!out || bins != c->plan.step_bins) return fail(c, EMT_ERR_INVALID_ARG, "bins must equal step_hist_bins");
    if (cudaSetDevice(c->opt.device) != cudaSuccess) return fail(c, EMT_ERR_CUDA, "cudaSetDevice");
    const size_t bytes = (size_t)3 * bins * sizeof(unsigned long long);
    EMT_CUDA(c, cudaMemcpyAsync(out, c->pool + c->plan.step_hist, bytes, cudaMemcpyDeviceToHost, c->stream));
    if (reset) EMT_CUDA(c, cudaMemsetAsync(c->pool + c->plan.step_hist, 0, bytes, c->stream));
    EMT_CUDA(c, cudaStreamSynchronize(c->stream));
    return EMT_OK;
}

emt_status emt_poll(emt_ctx* c, uint64_t* done_ids, int32_t cap, int32_t* n_done)
{
    emt_status r = check_ready(c);
    if (r != EMT_OK) return r;
    if (!n_done || (cap > 0 && !done_ids)) return fail(c, EMT_ERR_INVALID_ARG, "null output");
    r = drain_done(c);
    if (r != EMT_OK) return r;
    int k = 0;
    for (int s : c->order) {
        if (c->slot_state[s] == 2) {
            if (k < cap) done_ids[k] = c->slot_id[s];
            ++k;
        }
    }
    *n_done = std::min(k, cap);
    return EMT_OK;
}

emt_status emt_read_event(emt_ctx* c, uint64_t id, double* hist, double* summary)
{
    emt_status r = check_ready(c);
    if (r != EMT_OK) return r;
    auto f = c->id_to_slot.find(id);
    if (f == c->id_to_slot.end()) return fail(c, EMT_ERR_INVALID_ARG, "unknown event id");
    int s = f->second;
    if (c->slot_state[s] != 2) {
        r = drain_done(c);
        if (r != EMT_OK) return r;
        if (c->slot_state[s] != 2) return fail(c, EMT_ERR_NOT_READY, "event not finished");
    }
    const Plan& pl = c->plan;
    uint32_t slot = (uint32_t)s;
    EMT_CUDA(c, cudaMemcpyAsync(c->pool + pl.slots_tmp, &slot, 4, cudaMemcpyHostToDevice, c->stream));
    k_gather<<<1, 32, 0, c->stream>>>(c->at<uint32_t>(pl.slots_tmp), 1, c->at<double>(pl.hist), pl.hstride, c->n_bins,
                                      c->at<double>(pl.ledger), c->at<unsigned long long>(pl.counts),
                                      c->at<double>(pl.out_hist), c->at<double>(pl.out_summary));
    EMT_CUDA(c, cudaGetLastError());
    if (hist)
        EMT_CUDA(c, cudaMemcpyAsync(hist, c->pool + pl.out_hist, sizeof(double) * c->n_bins, cudaMemcpyDeviceToHost, c->stream));
    double sm[EMT_SUMMARY_LEN];
    EMT_CUDA(c, cudaMemcpyAsync(sm, c->pool + pl.out_summary, sizeof sm, cudaMemcpyDeviceToHost, c->stream));
    EMT_CUDA(c, cudaStreamSynchronize(c->stream));
    if (summary) std::memcpy(summary, sm, sizeof sm);
    c->order.erase(std::find(c->order.begin(), c->order.end(), s));
    release_slot(c, s);
    return EMT_OK;
}

emt_status emt_read_all(emt_ctx* c, double* hist, double* summary, uint64_t* ids, int32_t where)
{
    emt_status r = check_ready(c);
    if (r != EMT_OK) return r;
    if (in_flight(c) + on_host(c) != 0) return fail(c, EMT_ERR_NOT_READY, "tracks still in flight");
    if (where != EMT_HOST && where != EMT_DEVICE) return fail(c, EMT_ERR_INVALID_ARG, "where");
    const Plan& pl = c->plan;
    int n = (int)c->order.size();
    if (n == 0) return EMT_OK;
    std::vector<uint32_t> slots(c->order.begin(), c->order.end());
    EMT_CUDA(c, cudaMemcpyAsync(c->pool + pl.slots_tmp, slots.data(), 4 * (size_t)n, cudaMemcpyHostToDevice, c->stream));
    double* oh = where == EMT_DEVICE ? hist : c->at<double>(pl.out_hist);
    double* os = where == EMT_DEVICE ? summary : c->at<double>(pl.out_summary);
    if (where == EMT_DEVICE && !os) os = c->at<double>(pl.out_summary);
    k_gather<<<(n + 127) / 128, 128, 0, c->stream>>>(c->at<uint32_t>(pl.slots_tmp), n, c->at<double>(pl.hist), pl.hstride,
                                                     c->n_bins, c->at<double>(pl.ledger),
                                                     c->at<unsigned long long>(pl.counts), oh, os);
    EMT_CUDA(c, cudaGetLastError());
    if (where == EMT_HOST) {
        if (hist)
            EMT_CUDA(c, cudaMemcpyAsync(hist, oh, sizeof(double) * (size_t)n * c->n_bins, cudaMemcpyDeviceToHost, c->stream));
        if (summary)
            EMT_CUDA(c, cudaMemcpyAsync(summary, os, sizeof(double) * (size_t)n * EMT_SUMMARY_LEN, cudaMemcpyDeviceToHost,
                                        c->stream));
    }
    EMT_CUDA(c, cudaStreamSynchronize(c->stream));
    for (int k = 0; k < n; ++k) {
        if (ids) ids[k] = c->slot_id[slots[k]];
        release_slot(c, (int)slots[k]);
    }
    c->order.clear();
    return EMT_OK;
}

int32_t emt_events_in_flight(const emt_ctx* c) { return c ? (int32_t)c->order.size() : 0; }

int64_t emt_tracks_in_flight(const emt_ctx* c) { return c ? in_flight(c) + on_host(c) : 0; }

emt_status emt_get_table(emt_ctx* c, int32_t m, int32_t p, int32_t q, double* out, int32_t cap, int32_t* n_out)
{
    if (!c || !out || !n_out) return fail(c, EMT_ERR_INVALID_ARG, "null argument");
    if (!c->have_materials) return fail(c, EMT_ERR_BAD_STATE, "no tables");
    if (m < 0 || m >= c->n_mat || p < 0 || p > 2 || q < 0 || q > 5) return fail(c, EMT_ERR_INVALID_ARG, "table index");
    if (cap < c->n_grid) return fail(c, EMT_ERR_INVALID_ARG, "output too small");
    const Plan& pl = c->plan;
    std::vector<double> buf;
    if (q == 5) {
        EMT_CUDA(c, cudaMemcpy(out, c->pool + pl.grid, sizeof(double) * c->n_grid, cudaMemcpyDeviceToHost));
    } else if (q == 4) {
        EMT_CUDA(c, cudaMemcpy(out, c->pool + pl.dedx + sizeof(double) * (size_t)(m * 3 + p) * c->n_grid,
                               sizeof(double) * c->n_grid, cudaMemcpyDeviceToHost));
    } else {
        buf.resize((size_t)c->n_grid * kNq);
        EMT_CUDA(c, cudaMemcpy(buf.data(), c->pool + pl.tab + sizeof(double) * (size_t)(m * 3 + p) * c->n_grid * kNq,
                               sizeof(double) * buf.size(), cudaMemcpyDeviceToHost));
        for (int i = 0; i < c->n_grid; ++i) out[i] = buf[(size_t)i * kNq + q];
    }
    *n_out = c->n_grid;
    return EMT_OK;
}

emt_status emt_debug_set_tracks(emt_ctx* c, int32_t n, const double* rec, const uint64_t* uid, const int32_t* slot)
{
    emt_status r = check_ready(c);
    if (r != EMT_OK) return r;
    if (n < 0 || (n > 0 && (!rec || !uid || !slot))) return fail(c, EMT_ERR_INVALID_ARG, "bad arguments");
    if (c->plan.pipelined) return fail(c, EMT_ERR_BAD_STATE, "explicit track states need the fused or split schedule");
    if (n > c->plan.Q / 2) return fail(c, EMT_ERR_CAPACITY, "too many tracks");
    for (int i = 0; i < n; ++i) {
        int t = (int)rec[10 * (size_t)i], v = (int)rec[10 * (size_t)i + 8];
        if (t < 0 || t > 2 || v < -1 || v >= c->n_layers || slot[i] < 0 || slot[i] >= c->plan.max_events)
            return fail(c, EMT_ERR_INVALID_ARG, "bad track record");
    }
    const Plan& pl = c->plan;
    r = drain_done(c);  // injected tracks count toward their events again
    if (r != EMT_OK) return r;
    c->head_fresh = false;
    int cs = (int)(c->it % 3), side = (int)(c->it & 1);
    EMT_CUDA(c, cudaMemsetAsync(c->pool + pl.cnt + sizeof(Counters) * cs, 0, sizeof(Counters), c->stream));
    double* drec = nullptr;
    uint64_t* duid = nullptr;
    int32_t* dslot = nullptr;
    if (n > 0) {
        EMT_CUDA(c, cudaMalloc((void**)&drec, sizeof(double) * 10 * (size_t)n));
        EMT_CUDA(c, cudaMalloc((void**)&duid, sizeof(uint64_t) * (size_t)n));
        EMT_CUDA(c, cudaMalloc((void**)&dslot, sizeof(int32_t) * (size_t)n));
        EMT_CUDA(c, cudaMemcpyAsync(drec, rec, sizeof(double) * 10 * (size_t)n, cudaMemcpyHostToDevice, c->stream));
        EMT_CUDA(c, cudaMemcpyAsync(duid, uid, sizeof(uint64_t) * (size_t)n, cudaMemcpyHostToDevice, c->stream));
        EMT_CUDA(c, cudaMemcpyAsync(dslot, slot, sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, c->stream));
        cudaError_t e = c->mixed() ? Launch<float>::set_tracks(c->pf, side, cs, n, drec, duid, dslot, c->stream)
                                   : Launch<double>::set_tracks(c->pd, side, cs, n, drec, duid, dslot, c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "set tracks");
    }
    EMT_CUDA(c, cudaMemcpyAsync(c->h_cnt, c->pool + pl.cnt + sizeof(Counters) * cs, sizeof(Counters),
                                cudaMemcpyDeviceToHost, c->stream));
    EMT_CUDA(c, cudaStreamSynchronize(c->stream));
    cudaFree(drec);
    cudaFree(duid);
    cudaFree(dslot);
    c->live_g = c->h_cnt->n[0];
    c->live_c = c->h_cnt->n[1];
    return EMT_OK;
}

emt_status emt_debug_get_tracks(emt_ctx* c, int32_t cap, double* rec, uint64_t* uid, int32_t* slot, int32_t* n_out)
{
    emt_status r = check_ready(c);
    if (r != EMT_OK) return r;
    if (!n_out) return fail(c, EMT_ERR_INVALID_ARG, "null n_out");
    if (c->plan.pipelined) return fail(c, EMT_ERR_BAD_STATE, "explicit track states need the fused or split schedule");
    int n = (int)(c->live_g + c->live_c);
    *n_out = n;
    if (n == 0) return EMT_OK;
    if (cap < n || !rec || !uid || !slot) return fail(c, EMT_ERR_INVALID_ARG, "output too small");
    double* drec = nullptr;
    uint64_t* duid = nullptr;
    int32_t* dslot = nullptr;
    EMT_CUDA(c, cudaMalloc((void**)&drec, sizeof(double) * 10 * (size_t)n));
    EMT_CUDA(c, cudaMalloc((void**)&duid, sizeof(uint64_t) * (size_t)n));
    EMT_CUDA(c, cudaMalloc((void**)&dslot, sizeof(int32_t) * (size_t)n));
    int side = (int)(c->it & 1);
    cudaError_t e = c->mixed()
                        ? Launch<float>::get_tracks(c->pf, side, (int)c->live_g, (int)c->live_c, drec, duid, dslot, c->stream)
                        : Launch<double>::get_tracks(c->pd, side, (int)c->live_g, (int)c->live_c, drec, duid, dslot, c->stream);
    if (e != cudaSuccess) return cuda_fail(c, e, "get tracks");
    EMT_CUDA(c, cudaMemcpyAsync(rec, drec, sizeof(double) * 10 * (size_t)n, cudaMemcpyDeviceToHost, c->stream));
    EMT_CUDA(c, cudaMemcpyAsync(uid, duid, sizeof(uint64_t) * (size_t)n, cudaMemcpyDeviceToHost, c->stream));
    EMT_CUDA(c, cudaMemcpyAsync(slot, dslot, sizeof(int32_t) * (size_t)n, cudaMemcpyDeviceToHost, c->stream));
    EMT_CUDA(c, cudaStreamSynchronize(c->stream));
    cudaFree(drec);
    cudaFree(duid);
    cudaFree(dslot);
    return EMT_OK;
}

emt_status emt_debug_wait_timeout(int32_t device, int32_t timeout_ms)
{
    if (timeout_ms < 1 || timeout_ms > 60000) return EMT_ERR_INVALID_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return EMT_ERR_CUDA;
    int clock_khz = 0;
    if (cudaDeviceGetAttribute(&clock_khz, cudaDevAttrClockRate, device) != cudaSuccess || clock_khz < 1)
        return EMT_ERR_CUDA;
    char* buf = nullptr;
    cudaStream_t st = nullptr;
    emt_status rc = EMT_ERR_CUDA;
    int status = 0;
    const size_t bytes = 256 + sizeof(int);
    if (cudaMalloc(&buf, bytes) == cudaSuccess && cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) == cudaSuccess &&
        cudaMemsetAsync(buf, 0, bytes, st) == cudaSuccess &&
        launch_wait_never(reinterpret_cast<GridSync*>(buf), (long long)timeout_ms * clock_khz,
                          reinterpret_cast<int*>(buf + 256), 2, st) == cudaSuccess &&
        cudaMemcpyAsync(&status, buf + 256, sizeof(int), cudaMemcpyDeviceToHost, st) == cudaSuccess &&
        cudaStreamSynchronize(st) == cudaSuccess)
        rc = (status & kStatusTimeout) ? EMT_ERR_TIMEOUT : EMT_OK;
    if (st) cudaStreamDestroy(st);
    if (buf) cudaFree(buf);
    return rc;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Allocation-free entry point.  The paper has no counterpart: this exists
// for callers that must not allocate device memory (see include/emt.h).
// All device scratch (track buffers, counters, tables, geometry, scores)
// lives in one file-scope device array of kStaticPoolBytes.  Host code must
// not use the array's name as a device address: the address comes from
// cudaGetSymbolAddress, once per device, with that device current.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kStaticPoolBytes = (size_t)64 << 20;
__device__ __align__(256) unsigned char g_static_pool[kStaticPoolBytes];

constexpr int kStaticMaxDevices = 64;
std::mutex g_static_mutex;
void* g_static_ptr[kStaticMaxDevices] = {};

emt_options static_options(int32_t device, uint32_t seed)
{
    emt_options o;
    emt_default_options(&o);
    o.device = device;
    o.precision = EMT_PRECISION_FP64;
    o.slot_capacity = EMT_STATIC_MAX_TRACKS;
    o.max_events = EMT_STATIC_MAX_EVENTS;
    o.max_bins = EMT_STATIC_MAX_BINS;
    o.seed = seed;
    return o;
}

}  // namespace

extern "C" emt_status emt_transport_static(int32_t device, uint32_t seed, const emt_material* mats, int32_t n_mat,
                                           const emt_physics* ph, const emt_layer* layers, int32_t n_layers,
                                           const emt_world* w, int32_t n_events, const uint64_t* event_ids,
                                           const emt_primaries* prim, double* hist, double* summary,
                                           void* cuda_stream)
{
    // ---- arguments (sizes beyond the static limits are rejected)
    if (!mats || !ph || !layers || !w || !event_ids || !prim || !summary) return EMT_ERR_INVALID_ARG;
    if (n_events < 1 || n_events > EMT_STATIC_MAX_EVENTS) return EMT_ERR_CAPACITY;
    if (prim->n < 0 || prim->n > EMT_STATIC_MAX_PRIMARIES) return EMT_ERR_CAPACITY;
    if (w->n_bins < 1 || w->n_bins > EMT_STATIC_MAX_BINS) return EMT_ERR_CAPACITY;
    if (n_mat < 1 || n_mat > kMaxMat || n_layers < 1 || n_layers > kMaxLayers) return EMT_ERR_CAPACITY;
    if (prim->n > 0 && (!prim->event || !prim->type || !prim->T_MeV || !prim->pos_cm || !prim->dir))
        return EMT_ERR_INVALID_ARG;
    if (w->n_bins > 0 && !hist) return EMT_ERR_INVALID_ARG;
    if (!(ph->grid_lo_MeV > 0.0) || !(ph->grid_hi_MeV > ph->grid_lo_MeV) || ph->bins_per_decade < 1)
        return EMT_ERR_INVALID_ARG;
    const int n_grid = (int)std::floor(ph->bins_per_decade * std::log10(ph->grid_hi_MeV / ph->grid_lo_MeV) + 0.5) + 1;
    if (n_grid < 2 || n_grid > kMaxGrid) return EMT_ERR_INVALID_ARG;
    for (int k = 0; k < 3; ++k)
        if (!(ph->cut_MeV[k] > 0.0)) return EMT_ERR_INVALID_ARG;
    if (!(ph->step_frac > 0.0) || !(ph->final_range_cm > 0.0) || w->max_steps < 1) return EMT_ERR_INVALID_ARG;
    for (int e = 0; e < n_events; ++e)
        for (int f = e + 1; f < n_events; ++f)
            if (event_ids[e] == event_ids[f]) return EMT_ERR_INVALID_ARG;
    if (device < 0 || device >= kStaticMaxDevices) return EMT_ERR_INVALID_ARG;
    if (cudaSetDevice(device) != cudaSuccess) return EMT_ERR_CUDA;
    cudaStream_t st = (cudaStream_t)cuda_stream;

    // ---- device address of the static array (set-up, once per device)
    char* pool = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_static_mutex);
        if (!g_static_ptr[device]) {
            void* ptr = nullptr;
            if (cudaGetSymbolAddress(&ptr, g_static_pool) != cudaSuccess || !ptr) return EMT_ERR_CUDA;
            g_static_ptr[device] = ptr;
        }
        pool = (char*)g_static_ptr[device];
    }
    const emt_options opt = static_options(device, seed);
    const Plan pl = make_plan(opt);
    if (pl.total > kStaticPoolBytes) return EMT_ERR_CAPACITY;

    // ---- parameters pointing into the static array
    emt_ctx view;  // holds no resources: only the pool layout for fill_common
    view.opt = opt;
    view.plan = pl;
    view.pool = pool;
    Params<double> p;
    std::memset(&p, 0, sizeof p);
    fill_common(&view, p);

    // ---- zero what must start at zero (the array keeps the last call's data)
    if (cudaMemsetAsync(pool + pl.cnt, 0, pl.hist - pl.cnt, st) != cudaSuccess) return EMT_ERR_CUDA;
    if (cudaMemsetAsync(pool + pl.live, 0, pl.grid - pl.live, st) != cudaSuccess) return EMT_ERR_CUDA;

    // ---- materials and tables
    MaterialDev md[kMaxMat];
    double bk[kMaxMat];
    int vac[kMaxMat];
    for (int i = 0; i < n_mat; ++i) {
        const emt_material& m = mats[i];
        const bool vacuum = !(m.rho_g_cm3 > 0.0);
        if (!vacuum && (!(m.Z >= 1.0) || !(m.A_g_mol > 0.0) || !(m.I_eV > 0.0) || !(m.bk_MeV >= 0.0)))
            return EMT_ERR_INVALID_ARG;
        md[i] = {m.Z, m.A_g_mol, vacuum ? 0.0 : m.rho_g_cm3, m.I_eV, m.bk_MeV};
        bk[i] = m.bk_MeV;
        vac[i] = vacuum ? 1 : 0;
    }
    if (cudaMemcpyAsync(pool + pl.mats, md, sizeof(MaterialDev) * n_mat, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(pool + pl.bk, bk, sizeof(double) * n_mat, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(pool + pl.vacuum, vac, sizeof(int) * n_mat, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return EMT_ERR_CUDA;
    TableBuild b;
    b.mats = reinterpret_cast<const MaterialDev*>(pool + pl.mats);
    b.n_mat = n_mat;
    b.n_grid = n_grid;
    b.bpd = ph->bins_per_decade;
    b.e_lo = ph->grid_lo_MeV;
    for (int k = 0; k < 3; ++k) b.cut[k] = ph->cut_MeV[k];
    b.mask = ph->process_mask;
    b.x0 = reinterpret_cast<double*>(pool + pl.x0);
    b.ray_a = reinterpret_cast<double*>(pool + pl.ray_a);
    b.grid = reinterpret_cast<double*>(pool + pl.grid);
    b.tab = reinterpret_cast<double*>(pool + pl.tab);
    b.dedx = reinterpret_cast<double*>(pool + pl.dedx);
    b.tabf = nullptr;
    b.gridf = nullptr;
    b.igrid = reinterpret_cast<double*>(pool + pl.igrid);
    b.irs = reinterpret_cast<double*>(pool + pl.irs);
    b.igridf = nullptr;
    b.irsf = nullptr;
    b.dgrid = reinterpret_cast<double*>(pool + pl.dgrid);
    b.dtab = reinterpret_cast<double*>(pool + pl.dtab);
    b.dgridf = nullptr;
    b.dtabf = nullptr;
    if (build_tables(b, reinterpret_cast<double*>(pool + pl.scratch), st) != cudaSuccess) return EMT_ERR_CUDA;
    for (int k = 0; k < 3; ++k) {
        p.cut[k] = ph->cut_MeV[k];
        p.cutf[k] = (float)ph->cut_MeV[k];
    }
    p.grid = b.grid;
    p.tab = b.tab;
    p.igrid = b.igrid;
    p.irs = b.irs;
    p.dgrid = b.dgrid;
    p.dtab = b.dtab;
    p.n_grid = n_grid;
    p.bpd = ph->bins_per_decade;
    p.log10_lo = (float)std::log10(ph->grid_lo_MeV);
    p.step_frac = ph->step_frac;
    p.final_range = ph->final_range_cm;
    p.mask = ph->process_mask;
    p.step_fracf = (float)ph->step_frac;
    p.final_rangef = (float)ph->final_range_cm;

    // ---- geometry
    double zb[kMaxLayers + 1];
    int lm[kMaxLayers], lb[kMaxLayers];
    if (check_geometry(layers, n_layers, w, n_mat, EMT_STATIC_MAX_BINS, zb, lm, lb)) return EMT_ERR_INVALID_ARG;
    if (cudaMemcpyAsync(pool + pl.zb, zb, sizeof(double) * (n_layers + 1), cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(pool + pl.lmat, lm, sizeof(int) * n_layers, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(pool + pl.lbin, lb, sizeof(int) * n_layers, cudaMemcpyHostToDevice, st) != cudaSuccess)
        return EMT_ERR_CUDA;
    set_geometry(p, n_layers, w);

    // ---- events: slots 0..n_events-1 in order; primaries read in place
    uint32_t slots[EMT_STATIC_MAX_EVENTS];
    for (int e = 0; e < n_events; ++e) slots[e] = (uint32_t)e;
    if (cudaMemcpyAsync(pool + pl.st_slot, slots, 4 * (size_t)n_events, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemcpyAsync(pool + pl.st_ids, event_ids, 8 * (size_t)n_events, cudaMemcpyHostToDevice, st) != cudaSuccess ||
        cudaMemsetAsync(pool + pl.st_runs, 0, 4 * (size_t)n_events, st) != cudaSuccess)
        return EMT_ERR_CUDA;
    const int n = prim->n;
    int* status = reinterpret_cast<int*>(pool + pl.status);
    uint32_t* st_slot = reinterpret_cast<uint32_t*>(pool + pl.st_slot);
    if (n > 0) {
        k_runs<<<(n + 255) / 256, 256, 0, st>>>(prim->event, n, n_events, reinterpret_cast<uint32_t*>(pool + pl.st_start),
                                                reinterpret_cast<uint32_t*>(pool + pl.st_runs), status);
        k_uids<<<(n + 255) / 256, 256, 0, st>>>(prim->event, n, reinterpret_cast<uint32_t*>(pool + pl.st_start),
                                                reinterpret_cast<uint32_t*>(pool + pl.st_runs),
                                                reinterpret_cast<uint32_t*>(pool + pl.st_uid), status);
    }
    int h_status = 0;
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return EMT_ERR_CUDA;
    if (h_status != 0) return EMT_ERR_INVALID_ARG;
    k_reset_slots<<<(n_events + 127) / 128, 128, 0, st>>>(st_slot, n_events, p.hist, pl.hstride, p.ledger, p.counts,
                                                          p.live, reinterpret_cast<uint64_t*>(pool + pl.event_id),
                                                          reinterpret_cast<const uint64_t*>(pool + pl.st_ids));
    if (Launch<double>::admit(p, 0, 0, n, prim->event, prim->type, prim->T_MeV, prim->pos_cm, prim->dir, st_slot,
                              reinterpret_cast<const uint32_t*>(pool + pl.st_uid), st) != cudaSuccess)
        return EMT_ERR_CUDA;
    k_release_tokens<<<(n_events + 127) / 128, 128, 0, st>>>(st_slot, n_events, p.live, p.done_ring, p.done_head,
                                                             pl.max_events);
    if (cudaGetLastError() != cudaSuccess) return EMT_ERR_CUDA;

    // ---- admission outcome: a primary of an unknown particle type is the
    // caller's error, reported before any step runs
    Counters h_cnt;
    if (cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaMemcpyAsync(&h_cnt, pool + pl.cnt, sizeof h_cnt, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return EMT_ERR_CUDA;
    if (h_status & kStatusBadTrack) return EMT_ERR_INVALID_ARG;
    if (h_status != 0) return EMT_ERR_CUDA;

    // ---- step loop (host-driven; one counter read per step)
    int sms = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device);
    const int block = 256;
    const int resident = std::max(1, sms * Launch<double>::max_blocks_per_sm(block));
    int64_t live_g = h_cnt.n[0], live_c = h_cnt.n[1];
    unsigned long long steps[2] = {0, 0}, last_steps = 0;
    for (int64_t it = 0; live_g + live_c > 0; ++it) {
        const int side = (int)(it & 1), cin = (int)(it % 3), cout = (int)((it + 1) % 3), cclr = (int)((it + 2) % 3);
        const int64_t chunks = (live_g + block - 1) / block + (live_c + block - 1) / block;
        const int grid = (int)std::max<int64_t>(1, std::min<int64_t>(chunks, resident));
        if (Launch<double>::step(p, side, cin, cout, cclr, grid, block, st) != cudaSuccess) return EMT_ERR_CUDA;
        if (cudaMemcpyAsync(&h_cnt, pool + pl.cnt + sizeof(Counters) * ((it + 1) % 3), sizeof h_cnt,
                            cudaMemcpyDeviceToHost, st) != cudaSuccess ||
            cudaStreamSynchronize(st) != cudaSuccess)
            return EMT_ERR_CUDA;
        const bool same = live_g == h_cnt.n[0] && live_c == h_cnt.n[1];
        live_g = h_cnt.n[0];
        live_c = h_cnt.n[1];
        if (same && live_g + live_c > 0) {
            if (cudaMemcpyAsync(steps, pool + pl.total_steps, sizeof steps, cudaMemcpyDeviceToHost, st) != cudaSuccess ||
                cudaStreamSynchronize(st) != cudaSuccess)
                return EMT_ERR_CUDA;
            if (steps[0] == last_steps) return EMT_ERR_CAPACITY;
            last_steps = steps[0];
        }
    }

    // ---- results straight into the caller's device buffers
    k_gather<<<(n_events + 127) / 128, 128, 0, st>>>(st_slot, n_events, p.hist, pl.hstride, w->n_bins, p.ledger,
                                                     p.counts, hist, summary);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpyAsync(&h_status, status, sizeof(int), cudaMemcpyDeviceToHost, st) != cudaSuccess ||
        cudaStreamSynchronize(st) != cudaSuccess)
        return EMT_ERR_CUDA;
    return (h_status & (kStatusQueueOverflow | kStatusBadTrack)) ? EMT_ERR_CUDA : EMT_OK;
}
