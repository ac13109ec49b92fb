// Serving: fh_server_create / fh_submit / fh_poll with continuous batching.
//
// A scheduler thread owns the device side.  Each loop it
//   1. retires finished batches (event query, never a blocking wait): copies
//      each job's candidates out of the batch's pinned buffer, returns the
//      job's device bytes to the budget;
//   2. admits queued jobs in arrival order while their device bytes fit the
//      budget and a stream slot is free, and turns everything admitted at that
//      instant into ONE batch: per-job uploads and Doppler/position kernels,
//      one persistent transform launch over the tiles of all the batch's jobs
//      (up to kMaxBatchJobs per launch), per-job selection and a copy of the
//      candidates to pinned memory -- all on the slot's stream;
//   3. sleeps briefly when there is nothing to do.
// Jobs that arrive while earlier batches run form the next batch, which runs
// concurrently on another stream.  Device memory comes from the stream-ordered
// allocator (cudaMallocAsync / cudaFreeAsync), so admitting or retiring a job
// never synchronises the device.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "fh_internal.h"

using namespace fh;

namespace {

using Clock = std::chrono::steady_clock;

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

constexpr int32_t kServeWarps = 24;      // transform block size of served batches
constexpr int32_t kServePairWarps = 20;  // the same for batches of paired jobs

struct Job {
    fh_job_id id = 0;
    fh_plan_desc d{};
    double kt = 0.0;
    int32_t n_fft = 0, n_dir = 0, n_sb = 0;
    int64_t n_peaks = 0;
    std::vector<double> t, freq, v, sky;
    std::vector<int64_t> offsets;
    int64_t bytes = 0;
    int32_t state = FH_JOB_QUEUED;
    int32_t error = FH_OK;
    std::string message;
    std::vector<fh_candidate> result;
    double submit_s = 0, start_s = 0, done_s = 0;
    int32_t batch = -1, batch_jobs = 0;
    int32_t tile = 0;
    // device carve-up (valid while running)
    char *dbuf = nullptr;
    int64_t *d_off = nullptr, *d_S0 = nullptr, *d_D = nullptr, *d_A = nullptr;
    double *d_t = nullptr, *d_freq = nullptr, *d_v = nullptr, *d_sky = nullptr;
    uint64_t *d_prof = nullptr;
    fh_candidate *d_cand = nullptr;
    int32_t *d_err = nullptr;
    unsigned long long *d_dmax = nullptr;
    int32_t guard = 0;
    // what the job's items pair in the counters' 16-bit halves: 0 nothing, 1 two
    // directions, 2 (one direction) the two 32-row halves of 64-row slabs
    int32_t pairs = 0;
    uint32_t *d_win = nullptr;  // peak windows [unit][slab][tile][fft] at the job's tile
    int32_t *d_udelta = nullptr;  // (pairs == 1) per direction pair, the largest distance
    size_t pin_off = 0;  // offset of its candidates in the batch's pinned buffer
    size_t err_off = 0;

    int64_t cand_count() const { return (int64_t)n_dir * n_sb * d.top_k; }
    int32_t slab_rows() const { return pairs == 2 ? 2 * kRows : kRows; }
    int32_t n_slabs() const { return (d.n_fdot + slab_rows() - 1) / slab_rows(); }
    int32_t units() const { return pairs == 1 ? (n_dir + 1) / 2 : n_dir; }
    int32_t warps() const { return pairs ? kServePairWarps : kServeWarps; }
    int32_t n_tiles() const { return tile > 0 ? (d.n_f0 + tile - 1) / tile : 0; }

    // layout of the job's single device allocation
    int64_t layout(bool carve)
    {
        size_t o = 0;
        auto take = [&](size_t bytes) {
            const size_t at = o;
            o += align256(bytes > 0 ? bytes : 16);
            return at;
        };
        const size_t a_off = take(8 * ((size_t)n_fft + 1));
        const size_t a_t = take(8 * (size_t)n_fft);
        const size_t a_freq = take(8 * (size_t)n_peaks);
        const size_t a_v = take(24 * (size_t)n_fft);
        const size_t a_sky = take(24 * (size_t)n_dir);
        const size_t a_S0 = take(8 * (size_t)n_fft);
        const size_t a_D = take(8 * (size_t)n_fft);
        const size_t a_A = take(8 * (size_t)n_dir * (size_t)n_peaks);
        const size_t a_prof = take(8 * (size_t)n_dir * (size_t)d.n_f0);
        const size_t a_cand = take(sizeof(fh_candidate) * (size_t)cand_count());
        const size_t a_err = take(16);
        const size_t a_win = take(sizeof(uint32_t) * (size_t)units() * (size_t)n_slabs() *
                                  (size_t)n_tiles() * (size_t)std::max(1, n_fft));
        const size_t a_dmax = take(16);
        const size_t a_ud = take(pairs == 1 ? sizeof(int32_t) * (size_t)units() : 0);
        if (carve) {
            d_udelta = pairs == 1 ? (int32_t *)(dbuf + a_ud) : nullptr;
            d_dmax = (unsigned long long *)(dbuf + a_dmax);
            d_win = (uint32_t *)(dbuf + a_win);
            d_off = (int64_t *)(dbuf + a_off);
            d_t = (double *)(dbuf + a_t);
            d_freq = (double *)(dbuf + a_freq);
            d_v = (double *)(dbuf + a_v);
            d_sky = (double *)(dbuf + a_sky);
            d_S0 = (int64_t *)(dbuf + a_S0);
            d_D = (int64_t *)(dbuf + a_D);
            d_A = (int64_t *)(dbuf + a_A);
            d_prof = (uint64_t *)(dbuf + a_prof);
            d_cand = (fh_candidate *)(dbuf + a_cand);
            d_err = (int32_t *)(dbuf + a_err);
        }
        return (int64_t)o;
    }
};

struct Slot {
    cudaStream_t stream = nullptr;
    cudaEvent_t done = nullptr;
    unsigned int *sched = nullptr;  // the stream's transform item counter (zero between launches)
    char *pinned = nullptr;
    size_t pinned_bytes = 0;
    bool busy = false;
    int32_t batch = -1;
    std::vector<Job *> jobs;
};

}  // namespace

struct fh_server_s {
    int device = 0;
    int n_sm = 0;
    int64_t budget = 0;
    int64_t in_use = 0;
    cudaMemPool_t pool = nullptr;  // stream-ordered allocations of job buffers
    std::mutex mu;
    std::condition_variable cv;       // wakes the scheduler
    std::condition_variable done_cv;  // wakes drain()
    std::deque<Job *> queue;
    std::map<fh_job_id, std::unique_ptr<Job>> jobs;
    std::vector<Slot> slots;
    std::thread worker;
    bool stop = false;
    bool paused = false;
    int64_t next_id = 1;
    int32_t next_batch = 0;
    int64_t pending = 0;  // jobs not yet DONE/FAILED/CANCELLED
    Clock::time_point t0 = Clock::now();
    size_t prepared_smem = 0;
    std::string fatal;

    double now() const
    {
        return std::chrono::duration<double>(Clock::now() - t0).count();
    }
    void run();
    int launch_batch(Slot &slot, std::vector<Job *> &batch);
    void retire(Slot &slot);
    void fail_batch(Slot &slot, int code, const std::string &msg);
};

int fh_server_s::launch_batch(Slot &slot, std::vector<Job *> &batch)
{
    cudaStream_t s = slot.stream;
    // pinned space for candidates + error words
    size_t need = 0;
    for (Job *j : batch) {
        j->pin_off = need;
        need += align256(sizeof(fh_candidate) * (size_t)j->cand_count());
        j->err_off = need;
        need += 256;
    }
    if (need > slot.pinned_bytes) {
        if (slot.pinned) cudaFreeHost(slot.pinned);
        slot.pinned = nullptr;
        slot.pinned_bytes = 0;
        const size_t sz = std::max(need, (size_t)16 << 20);
        if (cudaMallocHost(&slot.pinned, sz) != cudaSuccess) {
            cudaGetLastError();
            return set_error(FH_ERR_NOMEM, "pinned buffer of %zu bytes", sz);
        }
        slot.pinned_bytes = sz;
    }
    cudaError_t e = cudaSuccess;
    for (Job *j : batch) {
        e = cudaMallocFromPoolAsync((void **)&j->dbuf, (size_t)j->bytes, pool, s);
        if (e != cudaSuccess) return cuda_error(e, "cudaMallocAsync(job)");
        j->layout(true);
        const fh_plan_desc &d = j->d;
        struct {
            void *dst;
            const void *src;
            size_t bytes;
        } cp[] = {{j->d_off, j->offsets.data(), 8 * ((size_t)j->n_fft + 1)},
                  {j->d_t, j->t.data(), 8 * (size_t)j->n_fft},
                  {j->d_freq, j->freq.data(), 8 * (size_t)j->n_peaks},
                  {j->d_v, j->v.data(), 24 * (size_t)j->n_fft},
                  {j->d_sky, j->sky.data(), 24 * (size_t)j->n_dir}};
        for (auto &c : cp)
            if (c.bytes && e == cudaSuccess)
                e = cudaMemcpyAsync(c.dst, c.src, c.bytes, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(j->d_err, 0, 16, s);
        if (e == cudaSuccess) e = cudaMemsetAsync(j->d_dmax, 0, 16, s);
        // shift tables and positions in one launch (the CSR was checked at submit)
        PrepArgs pa{};
        pa.offsets_in = nullptr;
        pa.offsets_out = j->d_off;
        pa.t = j->d_t;
        pa.v = j->d_v;
        pa.sky = j->d_sky;
        pa.n_fft = j->n_fft;
        pa.n_dir = j->n_dir;
        pa.n_fdot = d.n_fdot;
        pa.validate = 0;
        pa.n_peaks = j->n_peaks;
        pa.t_ref = d.t_ref;
        pa.kt = j->kt;
        pa.fdot_min = d.fdot_min;
        pa.fdot_step = d.fdot_step;
        pa.S0 = j->d_S0;
        pa.D = j->d_D;
        pa.dmax = j->d_dmax;
        pa.err = j->d_err;
        if (e == cudaSuccess) e = launch_correct(pa, j->d_freq, d.f0_min, d.k_over, j->d_A, nullptr, s);
        if (e == cudaSuccess)
            e = cudaMemsetAsync(j->d_prof, 0, 8 * (size_t)j->n_dir * d.n_f0, s);
        if (e != cudaSuccess) return cuda_error(e, "job set-up");
    }
    // One persistent transform launch per group of up to kMaxBatchJobs jobs.
    // A launch has one guard width (the largest its jobs need) and each job
    // keeps the tile its window table was sized for, so jobs (in order of
    // guard) join a group only while every member's tile still fits in shared
    // memory with the group's guard.
    // (a launch's jobs pair alike: grouped by what they pair, then by guard)
    const size_t lim = (size_t)max_optin_smem(device);
    std::vector<Job *> order(batch.begin(), batch.end());
    std::stable_sort(order.begin(), order.end(), [](const Job *x, const Job *y) {
        return x->pairs != y->pairs ? x->pairs < y->pairs : x->guard < y->guard;
    });
    for (size_t g = 0; g < order.size();) {
        const int32_t kind = order[g]->pairs;
        const int nwarps = order[g]->warps();
        auto fits = [&](const Job *j, int32_t guard) {
            return transform_smem_bytes(j->tile, j->d.k_over, FH_MODE_START, nwarps, guard) <= lim;
        };
        size_t g_end = g + 1;
        int32_t guard = std::max<int32_t>(2, order[g]->guard);
        while (g_end < order.size() && g_end - g < (size_t)kMaxBatchJobs &&
               order[g_end]->pairs == kind) {
            const int32_t gn = std::max(guard, order[g_end]->guard);
            bool ok = true;
            for (size_t k = g; k <= g_end && ok; ++k) ok = fits(order[k], gn);
            if (!ok) break;
            guard = gn;
            ++g_end;
        }
        JobTable tbl{};
        int64_t items = 0;
        size_t smem = 0;
        for (size_t k = g; k < g_end; ++k) {
            Job *j = order[k];
            TransformJob &t = tbl.job[tbl.n_jobs++];
            t.A = j->d_A;
            t.offsets = j->d_off;
            t.S0 = j->d_S0;
            t.D = j->d_D;
            t.profile = j->d_prof;
            t.maps = nullptr;
            t.dmax = j->d_dmax;
            t.err = j->d_err;
            t.weights = nullptr;  // served jobs use the plain map
            t.count_bound = j->n_peaks;
            t.n_peaks = j->n_peaks;
            t.n_fft = j->n_fft;
            t.n_f0 = j->d.n_f0;
            t.n_fdot = j->d.n_fdot;
            t.k_over = j->d.k_over;
            t.tile_cells = j->tile;
            t.n_slabs = j->n_slabs();
            t.n_tiles = j->n_tiles();
            t.dir_begin = 0;
            t.n_dir = j->n_dir;
            t.windows = j->d_win;
            t.dense = reinterpret_cast<int32_t *>(j->d_dmax + 1);  // beside dmax, cleared with it
            t.dir_pairs = j->pairs == 1 ? 1 : 0;
            t.row_pairs = j->pairs == 2 ? 1 : 0;
            t.unit_delta = j->d_udelta;
            t.delta_alloc = pair_delta(j->d);
            t.item_begin = items;
            t.n_items = (int64_t)t.n_slabs * t.n_tiles * j->units();
            if (j->d_udelta) {
                e = cudaMemsetAsync(j->d_udelta, 0, sizeof(int32_t) * (size_t)j->units(), s);
                if (e != cudaSuccess) return cuda_error(e, "cudaMemsetAsync(pair distances)");
            }
            items += t.n_items;
            smem = std::max(smem, transform_smem_bytes(j->tile, j->d.k_over, FH_MODE_START, nwarps,
                                                       guard));
            e = launch_windows(t, j->d_win, s);
            if (e != cudaSuccess) return cuda_error(e, "windows launch");
        }
        if (smem > prepared_smem) {
            e = transform_prepare(FH_MODE_START, smem);
            if (e != cudaSuccess) return cuda_error(e, "transform_prepare");
            prepared_smem = smem;
        }
        const int bps = std::max(1, transform_blocks_per_sm(FH_MODE_START, nwarps, smem));
        const int32_t grid = (int32_t)std::min<int64_t>(items, (int64_t)n_sm * bps);
        e = launch_transform(FH_MODE_START, tbl, items, grid, nwarps, smem, guard, s, slot.sched);
        if (e != cudaSuccess) return cuda_error(e, "transform launch");
        g = g_end;
    }
    for (Job *j : batch) {
        const fh_plan_desc &d = j->d;
        SelectArgs a{};
        a.profile = j->d_prof;
        a.out = j->d_cand;
        a.n_f0 = d.n_f0;
        a.subband_cells = d.subband_cells;
        a.top_k = d.top_k;
        a.excl = d.excl_cells;
        a.sep = d.sep_cells;
        a.n_thr = d.n_thr;
        a.n_sb = j->n_sb;
        a.dir_begin = 0;
        a.n_dir = j->n_dir;
        a.n_fft = j->n_fft;
        a.f0_min = d.f0_min;
        a.kt = j->kt;
        a.fdot_min = d.fdot_min;
        a.fdot_step = d.fdot_step;
        a.p0 = d.p0;
        e = launch_select(a, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(slot.pinned + j->pin_off, j->d_cand,
                                sizeof(fh_candidate) * (size_t)j->cand_count(),
                                cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(slot.pinned + j->err_off, j->d_err, 4, cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaFreeAsync(j->dbuf, s);
        if (e != cudaSuccess) return cuda_error(e, "job select/copy");
        j->dbuf = nullptr;
    }
    e = cudaEventRecord(slot.done, s);
    if (e != cudaSuccess) return cuda_error(e, "cudaEventRecord");
    return FH_OK;
}

void fh_server_s::retire(Slot &slot)
{
    const double t = now();
    for (Job *j : slot.jobs) {
        int32_t bits = 0;
        std::memcpy(&bits, slot.pinned + j->err_off, 4);
        if (bits) {
            j->state = FH_JOB_FAILED;
            j->error = bits & kErrRange ? FH_ERR_RANGE : FH_ERR_INVALID_ARG;
            j->message = "device-side check failed";
        } else {
            j->result.resize((size_t)j->cand_count());
            std::memcpy(j->result.data(), slot.pinned + j->pin_off,
                        sizeof(fh_candidate) * j->result.size());
            j->state = FH_JOB_DONE;
        }
        j->done_s = t;
        in_use -= j->bytes;
        --pending;
        // inputs are no longer needed
        std::vector<double>().swap(j->freq);
        std::vector<int64_t>().swap(j->offsets);
    }
    slot.jobs.clear();
    slot.busy = false;
}

void fh_server_s::fail_batch(Slot &slot, int code, const std::string &msg)
{
    const double t = now();
    for (Job *j : slot.jobs) {
        j->state = FH_JOB_FAILED;
        j->error = code;
        j->message = msg;
        j->done_s = t;
        in_use -= j->bytes;
        --pending;
    }
    slot.jobs.clear();
    slot.busy = false;
}

void fh_server_s::run()
{
    cudaSetDevice(device);
    std::unique_lock<std::mutex> lk(mu);
    for (;;) {
        bool progressed = false;
        // 1. retire
        for (Slot &sl : slots) {
            if (!sl.busy) continue;
            const cudaError_t q = cudaEventQuery(sl.done);
            if (q == cudaSuccess) {
                retire(sl);
                progressed = true;
            } else if (q != cudaErrorNotReady) {
                cudaGetLastError();
                fail_batch(sl, FH_ERR_CUDA, cudaGetErrorString(q));
                progressed = true;
            }
        }
        if (progressed) done_cv.notify_all();
        // 2. admit
        if (!paused && !queue.empty()) {
            Slot *free_slot = nullptr;
            for (Slot &sl : slots)
                if (!sl.busy) {
                    free_slot = &sl;
                    break;
                }
            if (free_slot) {
                std::vector<Job *> batch;
                while (!queue.empty() && in_use + queue.front()->bytes <= budget) {
                    Job *j = queue.front();
                    queue.pop_front();
                    in_use += j->bytes;
                    batch.push_back(j);
                }
                if (!batch.empty()) {
                    const int32_t b = next_batch++;
                    const double t = now();
                    for (Job *j : batch) {
                        j->state = FH_JOB_RUNNING;
                        j->start_s = t;
                        j->batch = b;
                        j->batch_jobs = (int32_t)batch.size();
                    }
                    free_slot->busy = true;
                    free_slot->batch = b;
                    free_slot->jobs = batch;
                    // the slot and its jobs belong to this thread until retired: launch
                    // without holding the lock so that submit/poll stay responsive
                    lk.unlock();
                    const int rc = launch_batch(*free_slot, batch);
                    lk.lock();
                    if (rc != FH_OK) {
                        // free whatever was allocated, stream-ordered, then fail the jobs
                        for (Job *j : batch)
                            if (j->dbuf) {
                                cudaFreeAsync(j->dbuf, free_slot->stream);
                                j->dbuf = nullptr;
                            }
                        cudaStreamSynchronize(free_slot->stream);
                        cudaGetLastError();
                        fail_batch(*free_slot, rc, fh_last_error());
                        done_cv.notify_all();
                    }
                    progressed = true;
                }
            }
        }
        bool busy = false;
        for (Slot &sl : slots) busy |= sl.busy;
        if (stop && !busy && (queue.empty() || paused)) break;
        if (!progressed) {
            if (busy)
                cv.wait_for(lk, std::chrono::microseconds(50));
            else
                cv.wait_for(lk, std::chrono::milliseconds(20));
        }
    }
}

namespace {

int copy_job(const fh_job_desc *jd, Job &j, int device)
{
    const fh_peakmap &pm = jd->peaks;
    if (pm.mem_kind != FH_MEM_HOST)
        return set_error(FH_ERR_INVALID_ARG, "served jobs take host-memory inputs");
    if (pm.n_fft < 0 || pm.n_peaks < 0 || jd->n_dir < 1 || jd->n_dir > 65535 || !jd->sky_n ||
        !pm.offsets)
        return set_error(FH_ERR_INVALID_ARG, "bad job sizes or null arrays");
    if (pm.n_peaks >= ((int64_t)1 << 31)) return set_error(FH_ERR_INVALID_ARG, "too many peaks");
    j.d = jd->plan;
    j.d.max_fft = std::max(1, pm.n_fft);
    j.d.max_dir = jd->n_dir;
    j.d.max_peaks = std::max<int64_t>(1, pm.n_peaks);
    j.d.mode = FH_MODE_START;
    j.d.schedule = FH_SCHED_BATCHED;
    int rc = validate_desc(j.d);
    if (rc) return rc;
    j.kt = (double)j.d.k_over * j.d.t_fft;
    rc = validate_host_inputs(j.d, j.kt, &pm, jd->v_over_c, jd->sky_n, jd->n_dir);
    if (rc) return rc;
    j.n_fft = pm.n_fft;
    j.n_peaks = pm.n_peaks;
    j.n_dir = jd->n_dir;
    j.n_sb = (j.d.n_f0 + j.d.subband_cells - 1) / j.d.subband_cells;
    j.t.assign(pm.t_fft, pm.t_fft + pm.n_fft);
    j.offsets.assign(pm.offsets, pm.offsets + pm.n_fft + 1);
    j.freq.assign(pm.freq, pm.freq + pm.n_peaks);
    j.v.assign(jd->v_over_c, jd->v_over_c + 3 * (size_t)pm.n_fft);
    j.sky.assign(jd->sky_n, jd->sky_n + 3 * (size_t)jd->n_dir);
    // the job runs with the library's default tile for its own guard cells
    const unsigned long long drift =
        std::max(default_drift(j.d), host_drift(j.d, j.kt, j.t.data(), j.n_fft));
    // pairs where they apply: two directions per item, or the row halves of one
    if (pairs_apply(j.d, device, j.n_fft, j.n_dir, drift)) {
        j.pairs = 1;
        j.guard = guard_for(drift) + pair_delta(j.d);
    } else if (rows_apply(j.d, device, j.n_fft, j.n_dir, drift)) {
        j.pairs = 2;
        j.guard = guard_for(drift, 2 * kRows - 1);
    } else {
        j.pairs = 0;
        j.guard = guard_for(drift);
    }
    j.tile = default_tile(j.d, device, FH_MODE_START, j.warps(), j.guard);
    j.bytes = j.layout(false);
    return FH_OK;
}

}  // namespace

extern "C" {

int fh_server_create(int64_t device_mem_budget, int32_t max_inflight, fh_server *out)
{
    if (!out) return set_error(FH_ERR_INVALID_ARG, "null out");
    *out = nullptr;
    if (device_mem_budget <= 0 || max_inflight < 1 || max_inflight > 64)
        return set_error(FH_ERR_INVALID_ARG, "budget must be > 0, max_inflight in [1, 64]");
    auto *sv = new (std::nothrow) fh_server_s;
    if (!sv) return set_error(FH_ERR_NOMEM, "host allocation failed");
    cudaError_t e = cudaGetDevice(&sv->device);
    if (e == cudaSuccess)
        e = cudaDeviceGetAttribute(&sv->n_sm, cudaDevAttrMultiProcessorCount, sv->device);
    sv->budget = device_mem_budget;
    if (e == cudaSuccess) {
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = sv->device;
        e = cudaMemPoolCreate(&sv->pool, &props);
        if (e == cudaSuccess) {
            uint64_t keep = (uint64_t)device_mem_budget;
            e = cudaMemPoolSetAttribute(sv->pool, cudaMemPoolAttrReleaseThreshold, &keep);
        }
    }
    sv->slots.resize((size_t)max_inflight);
    for (Slot &sl : sv->slots) {
        if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sl.stream, cudaStreamNonBlocking);
        if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sl.done, cudaEventDisableTiming);
        if (e == cudaSuccess) e = cudaMalloc(&sl.sched, 16);
        if (e == cudaSuccess) e = cudaMemset(sl.sched, 0, 16);
    }
    if (e != cudaSuccess) {
        for (Slot &sl : sv->slots) {
            if (sl.stream) cudaStreamDestroy(sl.stream);
            if (sl.done) cudaEventDestroy(sl.done);
            if (sl.sched) cudaFree(sl.sched);
        }
        if (sv->pool) cudaMemPoolDestroy(sv->pool);
        delete sv;
        return cuda_error(e, "fh_server_create");
    }
    sv->worker = std::thread([sv] { sv->run(); });
    *out = sv;
    return FH_OK;
}

int fh_server_destroy(fh_server sv)
{
    if (!sv) return FH_OK;
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        for (Job *j : sv->queue) {
            j->state = FH_JOB_CANCELLED;
            --sv->pending;
        }
        sv->queue.clear();
        sv->stop = true;
        sv->paused = false;
    }
    sv->cv.notify_all();
    // the scheduler exits once in-flight batches retire; wait for it, bounded
    const auto deadline = Clock::now() + std::chrono::seconds(60);
    bool finished = false;
    while (Clock::now() < deadline) {
        {
            std::lock_guard<std::mutex> lk(sv->mu);
            bool busy = false;
            for (Slot &sl : sv->slots) busy |= sl.busy;
            if (!busy) {
                finished = true;
                break;
            }
        }
        std::this_thread::sleep_for(std::chrono::milliseconds(1));
    }
    if (!finished) {
        // leave the server's memory alone: kernels may still use it
        sv->worker.detach();
        return set_error(FH_ERR_TIMEOUT, "in-flight batches did not finish within 60 s");
    }
    sv->worker.join();
    for (Slot &sl : sv->slots) {
        cudaStreamSynchronize(sl.stream);
        cudaStreamDestroy(sl.stream);
        cudaEventDestroy(sl.done);
        if (sl.sched) cudaFree(sl.sched);
        if (sl.pinned) cudaFreeHost(sl.pinned);
    }
    if (sv->pool) cudaMemPoolDestroy(sv->pool);
    delete sv;
    return FH_OK;
}

int fh_submit(fh_server sv, const fh_job_desc *jd, fh_job_id *out)
{
    if (!sv || !jd || !out) return set_error(FH_ERR_INVALID_ARG, "null server, job or out");
    auto job = std::make_unique<Job>();
    int rc = copy_job(jd, *job, sv->device);
    if (rc) return rc;
    std::lock_guard<std::mutex> lk(sv->mu);
    if (sv->stop) return set_error(FH_ERR_BAD_HANDLE, "server is shutting down");
    if (job->bytes > sv->budget)
        return set_error(FH_ERR_TOO_LARGE, "job needs %lld device bytes, budget is %lld",
                         (long long)job->bytes, (long long)sv->budget);
    job->id = sv->next_id++;
    job->submit_s = sv->now();
    *out = job->id;
    sv->queue.push_back(job.get());
    ++sv->pending;
    sv->jobs[job->id] = std::move(job);
    sv->cv.notify_all();
    return FH_OK;
}

int fh_poll(fh_server sv, fh_job_id id, int32_t *state, fh_candidate *out, int64_t capacity,
            int64_t *n_out)
{
    if (!sv || !state) return set_error(FH_ERR_INVALID_ARG, "null server or state");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->jobs.find(id);
    if (it == sv->jobs.end()) return set_error(FH_ERR_BAD_HANDLE, "unknown job %lld", (long long)id);
    Job &j = *it->second;
    *state = j.state;
    if (n_out) *n_out = j.cand_count();
    switch (j.state) {
    case FH_JOB_QUEUED:
    case FH_JOB_RUNNING:
        return FH_ERR_NOT_READY;
    case FH_JOB_CANCELLED:
        return set_error(FH_ERR_CANCELLED, "job %lld was cancelled", (long long)id);
    case FH_JOB_FAILED:
        return set_error(j.error, "job %lld failed: %s", (long long)id, j.message.c_str());
    default:
        break;
    }
    if (!out || capacity < (int64_t)j.result.size())
        return set_error(FH_ERR_CAPACITY, "need %lld candidate slots", (long long)j.result.size());
    std::memcpy(out, j.result.data(), sizeof(fh_candidate) * j.result.size());
    return FH_OK;
}

int fh_job_get_stats(fh_server sv, fh_job_id id, fh_job_stats *out)
{
    if (!sv || !out) return set_error(FH_ERR_INVALID_ARG, "null server or out");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->jobs.find(id);
    if (it == sv->jobs.end()) return set_error(FH_ERR_BAD_HANDLE, "unknown job %lld", (long long)id);
    const Job &j = *it->second;
    out->submit_s = j.submit_s;
    out->start_s = j.start_s;
    out->done_s = j.done_s;
    out->updates = (int64_t)j.n_dir * j.d.n_fdot * j.n_peaks;
    out->device_bytes = j.bytes;
    out->batch = j.batch;
    out->batch_jobs = j.batch_jobs;
    return FH_OK;
}

int fh_cancel(fh_server sv, fh_job_id id)
{
    if (!sv) return set_error(FH_ERR_INVALID_ARG, "null server");
    std::lock_guard<std::mutex> lk(sv->mu);
    auto it = sv->jobs.find(id);
    if (it == sv->jobs.end()) return set_error(FH_ERR_BAD_HANDLE, "unknown job %lld", (long long)id);
    Job *j = it->second.get();
    if (j->state != FH_JOB_QUEUED)
        return set_error(FH_ERR_INVALID_ARG, "job %lld is no longer queued", (long long)id);
    sv->queue.erase(std::remove(sv->queue.begin(), sv->queue.end(), j), sv->queue.end());
    j->state = FH_JOB_CANCELLED;
    j->done_s = sv->now();
    --sv->pending;
    sv->done_cv.notify_all();
    return FH_OK;
}

int fh_server_drain(fh_server sv, double timeout_s)
{
    if (!sv) return set_error(FH_ERR_INVALID_ARG, "null server");
    std::unique_lock<std::mutex> lk(sv->mu);
    const auto deadline = Clock::now() + std::chrono::duration_cast<Clock::duration>(
                                             std::chrono::duration<double>(std::max(0.0, timeout_s)));
    while (sv->pending > 0) {
        if (sv->done_cv.wait_until(lk, deadline) == std::cv_status::timeout && sv->pending > 0)
            return set_error(FH_ERR_TIMEOUT, "%lld jobs still pending", (long long)sv->pending);
    }
    return FH_OK;
}

int fh_server_pause(fh_server sv, int32_t paused)
{
    if (!sv) return set_error(FH_ERR_INVALID_ARG, "null server");
    {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->paused = paused != 0;
    }
    sv->cv.notify_all();
    return FH_OK;
}

}  // extern "C"
