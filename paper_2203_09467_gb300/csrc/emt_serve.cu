// emt_serve.cu -- event-request serving loop on top of the public C ABI.
//
// The paper asks for many concurrent events to fill the device (Sec. 2.4;
// Sec. 3.2: workflows will have to group several events into one batch).  Two schedules over one context (whose track state stays on
// the device across requests):
//   continuous : requests that arrive while others are in flight are
//                admitted as soon as event slots and track slots allow
//                and fewer than admit_below tracks are in flight (growing
//                showers need room: a full track store can only defer);
//                the step loop advances a few iterations between
//                admissions, and finished events are read back at once.
//   batch      : one batch at a time: when the device is idle, every
//                request that has arrived is admitted together and run to
//                completion before the next batch starts.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <thread>
#include <vector>

#include "../../include/emt.h"

namespace {

using Clock = std::chrono::steady_clock;

double seconds_since(Clock::time_point t0)
{
    return std::chrono::duration<double>(Clock::now() - t0).count();
}

}  // namespace

extern "C" emt_status emt_serve(emt_ctx* ctx, int32_t n_events, const uint64_t* event_ids, const double* arrival_s,
                                const int32_t* first, const int32_t* count, const emt_primaries* prim,
                                const emt_serve_options* opt, double* admit_s, double* done_s, double* hist,
                                double* summary)
{
    if (!ctx || n_events < 1 || !event_ids || !arrival_s || !first || !count || !prim || !opt || !done_s)
        return EMT_ERR_INVALID_ARG;
    if (opt->mode != EMT_SERVE_CONTINUOUS && opt->mode != EMT_SERVE_BATCH) return EMT_ERR_INVALID_ARG;
    if (!(opt->time_scale > 0.0) || opt->steps_per_poll < 1 || opt->n_bins < 0) return EMT_ERR_INVALID_ARG;
    for (int e = 0; e < n_events; ++e) {
        if (count[e] < 0 || first[e] < 0 || first[e] + count[e] > prim->n) return EMT_ERR_INVALID_ARG;
        if (e > 0 && arrival_s[e] < arrival_s[e - 1]) return EMT_ERR_INVALID_ARG;
    }
    const int nb = opt->n_bins;
    std::vector<int32_t> ev_idx;
    std::vector<uint64_t> ids;
    std::vector<uint64_t> done_ids(std::max(1, n_events));
    std::vector<int> index_of_slot;  // position in the request list, by order of admission
    std::vector<double> h(std::max(1, nb)), sm(EMT_SUMMARY_LEN);
    // map event id -> request index (ids are distinct)
    std::vector<std::pair<uint64_t, int>> id_index(n_events);
    for (int e = 0; e < n_events; ++e) id_index[e] = {event_ids[e], e};
    std::sort(id_index.begin(), id_index.end());
    auto index_of = [&](uint64_t id) {
        auto it = std::lower_bound(id_index.begin(), id_index.end(), std::make_pair(id, -1));
        return (it != id_index.end() && it->first == id) ? it->second : -1;
    };
    // submit requests [a, b) as one call
    auto submit_range = [&](int a, int b) -> emt_status {
        int np = 0;
        for (int e = a; e < b; ++e) np += count[e];
        ev_idx.resize(std::max(np, 1));
        ids.resize(b - a);
        int k = 0;
        for (int e = a; e < b; ++e) {
            ids[e - a] = event_ids[e];
            for (int j = 0; j < count[e]; ++j) ev_idx[k++] = e - a;
        }
        emt_primaries sub;
        sub.n = np;
        sub.event = ev_idx.data();
        const int f = first[a];
        // requests are contiguous in the primary arrays: [first[a], first[b-1] + count[b-1])
        sub.type = prim->type + f;
        sub.T_MeV = prim->T_MeV + f;
        sub.pos_cm = prim->pos_cm + 3 * (size_t)f;
        sub.dir = prim->dir + 3 * (size_t)f;
        return emt_submit(ctx, b - a, ids.data(), &sub, EMT_HOST);
    };
    auto finish = [&](uint64_t id, double t) -> emt_status {
        int e = index_of(id);
        if (e < 0) return EMT_ERR_INVALID_ARG;
        emt_status r = emt_read_event(ctx, id, nb > 0 ? h.data() : nullptr, sm.data());
        if (r != EMT_OK) return r;
        done_s[e] = t;
        if (hist && nb > 0) std::memcpy(hist + (size_t)e * nb, h.data(), sizeof(double) * nb);
        if (summary) std::memcpy(summary + (size_t)e * EMT_SUMMARY_LEN, sm.data(), sizeof(double) * EMT_SUMMARY_LEN);
        return EMT_OK;
    };
    for (int e = 1; e < n_events; ++e)
        if (first[e] != first[e - 1] + count[e - 1]) return EMT_ERR_INVALID_ARG;

    const Clock::time_point t0 = Clock::now();
    const double scale = opt->time_scale;
    int next = 0;      // first request not admitted yet
    int finished = 0;  // requests done
    while (finished < n_events) {
        const double now = seconds_since(t0);
        int arrived = next;
        while (arrived < n_events && arrival_s[arrived] / scale <= now) ++arrived;
        const bool idle = emt_events_in_flight(ctx) == 0;
        const bool room = opt->admit_below <= 0 || emt_tracks_in_flight(ctx) < opt->admit_below;
        if (next < arrived && (idle || (opt->mode == EMT_SERVE_CONTINUOUS && room))) {
            // admit as many arrived requests as fit, halving on capacity errors
            int want = arrived - next;
            while (want > 0) {
                emt_status r = submit_range(next, next + want);
                if (r == EMT_OK) {
                    const double ta = seconds_since(t0);
                    for (int e = next; e < next + want; ++e)
                        if (admit_s) admit_s[e] = ta;
                    next += want;
                    break;
                }
                if (r != EMT_ERR_CAPACITY) return r;
                want /= 2;
            }
        }
        if (emt_events_in_flight(ctx) == 0) {
            if (next >= n_events) break;
            // nothing to do until the next arrival
            const double wait = arrival_s[next] / scale - seconds_since(t0);
            if (wait > 0) std::this_thread::sleep_for(std::chrono::duration<double>(wait));
            continue;
        }
        emt_run_stats st;
        emt_status r = emt_run(ctx, opt->mode == EMT_SERVE_CONTINUOUS ? opt->steps_per_poll : 0, &st);
        if (r != EMT_OK) return r;
        int32_t nd = 0;
        r = emt_poll(ctx, done_ids.data(), n_events, &nd);
        if (r != EMT_OK) return r;
        const double td = seconds_since(t0);
        for (int k = 0; k < nd; ++k) {
            r = finish(done_ids[k], td);
            if (r != EMT_OK) return r;
            ++finished;
        }
    }
    return finished == n_events ? EMT_OK : EMT_ERR_BAD_STATE;
}
