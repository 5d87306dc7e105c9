// sell_server.cu -- continuous-batching SpMV/SpMMV server over device-resident
// SELL-C-sigma matrices (an extension: the paper stops at single products).
//
// Requests (matrix, block of right-hand sides in pinned host memory) arrive at
// any time from any thread.  One scheduler thread per server:
//   * admits queued requests in arrival order while their device footprint
//     (x block, y block, long-row scratch) fits in an arena of
//     budget - resident bytes -- the HBM budget is never exceeded;
//   * packs the admitted ones into one batch plan (sell_batch.cu: one launch
//     per kernel variant, every product bitwise the same as alone) on a free
//     stream, with the device-to-host copies of the results after it;
//   * meters the host-to-device copies of the x blocks itself: copies on
//     different streams share the copy engine first in, first out (a 64 KB
//     copy issued after a 256 MB one on another stream finishes with it,
//     1.3 ms later), so every input goes through one copy stream in chunks
//     of kChunk bytes, at most kWindow bytes in flight, the batch with the
//     fewest bytes left first, where a waiting batch's count falls at
//     kAgeRate bytes per second of its age (a large input is not starved by
//     a stream of small ones: it waits about its own copy time at most
//     before it goes first); a batch's kernels are enqueued behind an event
//     recorded after its last chunk.  A small request then waits for at
//     most a window of chunks, or one aged large input, instead of every
//     large input issued before it;
//   * runs a batch in two parts when its products differ widely in size:
//     the requests whose work is at most 1/kPartRatio of the batch's largest
//     go first, with their own input copies, plan and completion event, so
//     they complete without waiting for the large products of their batch;
//   * keeps up to `streams` batches in flight, so requests that arrive while
//     others run are admitted as soon as a stream and memory are free and
//     their work overlaps on the device;
//   * retires a batch when its completion event has passed: stamps the
//     requests, returns their memory to the arena and wakes their waiters.
// Times are seconds on a steady clock shared by all requests of the process.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "sell_arena.h"
#include "sell_internal.cuh"

namespace sell {
namespace {

double now_s() {
    using namespace std::chrono;
    return duration<double>(steady_clock::now().time_since_epoch()).count();
}

enum ReqState { kQueued = 0, kRunning = 1, kDone = 2 };

struct Req {
    uint64_t id = 0;
    int32_t mid = 0, k = 1;
    uint32_t flags = 0;
    const void *X = nullptr;  // host
    void *Y = nullptr;        // host, or null: the result stays on the device
    size_t xb = 0, yb = 0, sb = 0, xoff = 0, yoff = 0, soff = 0;
    bool reserved = false;
    double ta = 0, tl = 0, td = 0;
    int state = kQueued;
    int32_t status = SELL_OK, batch = 0;
    bool collected = false;  // delivered by sell_server_wait or sell_server_next
    bool keep_y() const { return Y == nullptr; }
};

// Input copies are issued in chunks of at most kChunk bytes, at most
// kWindow bytes in flight on the copy stream (about 160 us at 200 GB/s).
constexpr size_t kChunk = 4u << 20;
constexpr size_t kWindow = 32u << 20;
// The copy order's aging: a part's bytes left, less its age times this rate
// (about the copy engine's host-to-device rate), picks the next chunk.
// Plain fewest-bytes-left-first starved large inputs: under Poisson load
// parts of 0.25-1 GB waited 50-170 ms for their chunks to be issued (then
// copied in a few ms) while smaller parts kept arriving.
constexpr double kAgeRate = 200e9;

struct Chunk {
    char *dst;
    const char *src;
    size_t bytes;
};

// A request is in the first part of its batch when its work is at most
// 1/kPartRatio of the batch's largest request.
constexpr double kPartRatio = 8.0;

// One part of a batch: its requests, their input copies, its plan.
struct Part {
    sell_batch *plan = nullptr;
    std::vector<Req *> reqs;
    std::vector<Chunk> chunks;  // its host-to-device copies, in order
    size_t next = 0;            // the next chunk to issue
    size_t left = 0;            // bytes not yet issued
    bool launched = false;      // kernels, result copies and completion event enqueued
    bool retired = false;       // its requests are done
    sell_status status = SELL_OK;
    double t_admit = 0;         // when its batch was admitted (the copy order's age)
};

// A batch holds one stream; its parts run on it in order (part 0 first).
struct Batch {
    int si = 0;
    int nparts = 1;
    Part parts[2];
};

bool is_pinned_host(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        (void)cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

}  // namespace
}  // namespace sell

struct sell_server {
    std::vector<sell_matrix *> mats;
    int device = 0;
    int64_t budget = 0, resident = 0, arena_bytes = 0, used = 0, peak_used = 0;
    int32_t max_batch = 64, nstreams = 3, size_ratio = 0;
    int64_t max_work = 0;  // cap on a batch's work (stored elements x k), 0: none
    sell::Allocator al;
    char *arena_base = nullptr;
    sell::Arena arena;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> events;  // two per stream (a stream holds at most one batch): its parts done
    std::vector<cudaEvent_t> ready;   // two per stream: each part's input copies issued (on h2d)
    cudaStream_t h2d = nullptr;       // the copy stream of every input
    std::deque<std::pair<cudaEvent_t, size_t>> copying;  // chunks in flight on h2d (event after each)
    std::vector<cudaEvent_t> spare;   // chunk events to reuse
    size_t copy_bytes = 0;            // bytes in flight on h2d
    std::deque<int> free_streams;
    std::vector<sell::Batch> inflight;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::deque<sell::Req *> queue;
    std::unordered_map<uint64_t, sell::Req *> reqs;
    std::deque<uint64_t> completed;  // in completion order, for sell_server_next
    uint64_t next_id = 1;
    int64_t nreq = 0, nbatch = 0, nbatched = 0;
    bool stop = false;
    std::thread thr;
};

namespace sell {
namespace {

// Device footprint of a request: its x and y blocks and its long-row scratch.
void sizes(const sell_server *S, Req *r) {
    const sell_matrix *h = S->mats[r->mid];
    const size_t es = h->store_type == SELL_F64 ? 8 : 4;
    r->xb = (size_t)h->ncols * r->k * es;
    r->yb = (size_t)h->nrows * r->k * es;
    r->sb = batch_item_scratch(h, r->k, r->flags, nullptr);
}

// Work of a request: stored elements times right-hand sides.
double work(const sell_server *S, const Req *r) { return (double)S->mats[r->mid]->stored * r->k; }

size_t footprint(const Req *r) { return region(r->xb) + region(r->yb) + (r->sb ? round256(r->sb) : 0); }

bool reserve(sell_server *S, Req *r) {
    size_t xo = 0, yo = 0, so = 0;
    if (!S->arena.alloc(region(r->xb), &xo)) return false;
    if (!S->arena.alloc(region(r->yb), &yo)) {
        S->arena.release(xo, region(r->xb));
        return false;
    }
    if (r->sb && !S->arena.alloc(r->sb, &so)) {
        S->arena.release(xo, region(r->xb));
        S->arena.release(yo, region(r->yb));
        return false;
    }
    r->xoff = xo;
    r->yoff = yo;
    r->soff = so;
    r->reserved = true;
    S->used += (int64_t)footprint(r);
    S->peak_used = std::max(S->peak_used, S->used);
    return true;
}

void release_x_s(sell_server *S, Req *r) {
    S->arena.release(r->xoff, region(r->xb));
    S->used -= (int64_t)region(r->xb);
    if (r->sb) {
        S->arena.release(r->soff, r->sb);
        S->used -= (int64_t)round256(r->sb);
    }
}

void release_y(sell_server *S, Req *r) {
    S->arena.release(r->yoff, region(r->yb));
    S->used -= (int64_t)region(r->yb);
    r->reserved = false;
}

// Admit a batch on stream si: stamp its requests, split it into parts and
// list each part's input copies in chunks (no CUDA call; the scheduler
// thread owns the batch from here).
void prepare(sell_server *S, int si, std::vector<Req *> &batch, Batch &B) {
    const double t = now_s();
    const int n = (int)batch.size();
    B.si = si;
    double wmax = 0;
    for (Req *r : batch) wmax = std::max(wmax, work(S, r));
    int nsmall = 0;
    for (Req *r : batch) nsmall += work(S, r) * kPartRatio <= wmax ? 1 : 0;
    B.nparts = (nsmall > 0 && nsmall < n) ? 2 : 1;
    for (int i = 0; i < n; ++i) {
        Req *r = batch[i];
        r->tl = t;
        r->batch = n;
        const int p = (B.nparts == 2 && work(S, r) * kPartRatio > wmax) ? 1 : 0;
        Part &P = B.parts[p];
        P.t_admit = t;
        P.reqs.push_back(r);
        auto add = [&](char *dst, const void *src, size_t bytes) {
            const char *s = static_cast<const char *>(src);
            for (size_t o = 0; o < bytes; o += kChunk) {
                const size_t c = std::min(kChunk, bytes - o);
                P.chunks.push_back({dst + o, s + o, c});
                P.left += c;
            }
        };
        if (r->xb) add(S->arena_base + r->xoff, r->X, r->xb);
        if ((r->flags & SELL_SPMV_ACCUMULATE) && r->yb) add(S->arena_base + r->yoff, r->Y, r->yb);
    }
}

// Enqueue a part whose input copies have all been issued: its stream waits
// for them, then runs the part's plan, its result copies and its completion
// event (called without the lock).
void finish_launch(sell_server *S, Batch &B, int p) {
    Part &P = B.parts[p];
    const int si = B.si;
    cudaStream_t st = S->streams[si];
    cudaEvent_t ready = S->ready[2 * si + p], done = S->events[2 * si + p];
    const int n = (int)P.reqs.size();
    sell_status status = P.status;
    if (status == SELL_OK && !P.chunks.empty() &&
        (cudaEventRecord(ready, S->h2d) != cudaSuccess || cudaStreamWaitEvent(st, ready, 0) != cudaSuccess))
        status = cuda_fail(cudaGetLastError(), "server: input copy ordering");
    std::vector<sell_batch_item> items(n);
    std::vector<void *> scr(n, nullptr);
    for (int i = 0; i < n; ++i) {
        Req *r = P.reqs[i];
        items[i].A = S->mats[r->mid];
        items[i].X = S->arena_base + r->xoff;
        items[i].Y = S->arena_base + r->yoff;
        items[i].ldx = r->k;
        items[i].ldy = r->k;
        items[i].k = r->k;
        items[i].flags = r->flags;
        scr[i] = r->sb ? S->arena_base + r->soff : nullptr;
    }
    if (status == SELL_OK) {
        P.plan = new (std::nothrow) sell_batch();
        if (!P.plan) status = SELL_ENOMEM;
    }
    if (status == SELL_OK) status = batch_create(items.data(), n, st, P.plan, scr.data());
    if (status == SELL_OK) status = batch_run(P.plan, 0, st);
    for (int i = 0; i < n && status == SELL_OK; ++i) {
        Req *r = P.reqs[i];
        if (!r->keep_y() && r->yb &&
            cudaMemcpyAsync(r->Y, S->arena_base + r->yoff, r->yb, cudaMemcpyDeviceToHost, st) != cudaSuccess)
            status = cuda_fail(cudaGetLastError(), "server: result copy");
    }
    if (status != SELL_OK)
        for (Req *r : P.reqs) r->status = status;
    if (cudaEventRecord(done, st) != cudaSuccess) {
        (void)cudaGetLastError();
        (void)cudaStreamSynchronize(st);
    }
    P.launched = true;
}

// Feed the copy stream (called without the lock, scheduler thread only):
// retire the chunks that have landed, launch the parts whose copies are all
// issued (a batch's second part after its first), and issue further chunks
// while the window has room -- always from the part with the fewest bytes
// left less kAgeRate times its age (the earliest admitted on ties).
void pump(sell_server *S) {
    while (!S->copying.empty()) {
        const cudaError_t q = cudaEventQuery(S->copying.front().first);
        if (q == cudaErrorNotReady) break;
        if (q != cudaSuccess) (void)cudaGetLastError();  // the part's own event reports the failure
        S->copy_bytes -= S->copying.front().second;
        S->spare.push_back(S->copying.front().first);
        S->copying.pop_front();
    }
    const double now = now_s();
    for (;;) {
        Part *pick = nullptr;
        double best = 0;
        for (Batch &B : S->inflight) {
            for (int p = 0; p < B.nparts; ++p) {
                Part &P = B.parts[p];
                if (P.launched) continue;
                if (p > 0 && !B.parts[p - 1].launched) break;  // parts launch in order
                if (P.next == P.chunks.size()) {
                    finish_launch(S, B, p);
                    continue;
                }
                const double key = (double)P.left - (now - P.t_admit) * kAgeRate;
                if (!pick || key < best) {
                    pick = &P;
                    best = key;
                }
            }
        }
        if (!pick || S->copy_bytes >= kWindow) return;
        const Chunk &c = pick->chunks[pick->next];
        cudaEvent_t ev = nullptr;
        if (!S->spare.empty()) {
            ev = S->spare.back();
            S->spare.pop_back();
        } else if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) {
            ev = nullptr;
        }
        if (!ev || cudaMemcpyAsync(c.dst, c.src, c.bytes, cudaMemcpyHostToDevice, S->h2d) != cudaSuccess ||
            cudaEventRecord(ev, S->h2d) != cudaSuccess) {
            pick->status = cuda_fail(cudaGetLastError(), "server: input copy");
            if (ev) S->spare.push_back(ev);
            pick->next = pick->chunks.size();  // no further copies; the part reports the failure
            pick->left = 0;
            continue;
        }
        S->copying.push_back({ev, c.bytes});
        S->copy_bytes += c.bytes;
        pick->next += 1;
        pick->left -= c.bytes;
    }
}

void scheduler(sell_server *S) {
    (void)cudaSetDevice(S->device);
    std::unique_lock<std::mutex> lk(S->mu);
    for (;;) {
        // retire finished batches
        bool retired = false;
        for (size_t i = 0; i < S->inflight.size();) {
            Batch &B = S->inflight[i];
            bool all = true;
            for (int p = 0; p < B.nparts; ++p) {
                Part &P = B.parts[p];
                if (P.retired) continue;
                if (!P.launched) {  // still waiting for its input copies
                    all = false;
                    continue;
                }
                const cudaError_t q = cudaEventQuery(S->events[2 * B.si + p]);
                if (q == cudaErrorNotReady) {
                    all = false;
                    continue;
                }
                if (q != cudaSuccess) (void)cudaGetLastError();
                const double t = now_s();
                for (Req *r : P.reqs) {
                    r->td = t;
                    if (q != cudaSuccess && r->status == SELL_OK) r->status = SELL_ECUDA;
                    release_x_s(S, r);
                    if (!r->keep_y() || r->status != SELL_OK) release_y(S, r);
                    r->state = kDone;
                    S->completed.push_back(r->id);
                }
                if (P.plan) {
                    batch_release(P.plan, S->streams[B.si]);
                    delete P.plan;
                    P.plan = nullptr;
                }
                P.retired = true;
                retired = true;
            }
            if (!all) {
                ++i;
                continue;
            }
            S->free_streams.push_back(B.si);
            S->inflight.erase(S->inflight.begin() + i);
        }
        if (retired) S->cv_done.notify_all();
        // admit in arrival order while the footprint fits, then launch.  With
        // a size ratio, the batch takes the oldest request and then, among the
        // next requests in order, those whose work is within the ratio of it
        // (the others wait for the next batch, on another stream), so small
        // requests do not wait for the end of a large one's launch.
        while (!S->free_streams.empty() && !S->queue.empty()) {
            std::vector<Req *> batch;
            if (S->size_ratio <= 1) {
                double bw = 0;  // the batch's work so far
                while (!S->queue.empty() && (int)batch.size() < S->max_batch) {
                    Req *r = S->queue.front();
                    const double w = work(S, r);
                    if (!batch.empty() && S->max_work > 0 && bw + w > (double)S->max_work) break;
                    if (!reserve(S, r)) break;
                    S->queue.pop_front();
                    r->state = kRunning;
                    batch.push_back(r);
                    bw += w;
                }
            } else {
                Req *head = S->queue.front();
                if (reserve(S, head)) {
                    S->queue.pop_front();
                    head->state = kRunning;
                    batch.push_back(head);
                    const double w0 = work(S, head), q = (double)S->size_ratio;
                    size_t scan = std::min(S->queue.size(), (size_t)4 * S->max_batch);
                    for (size_t i = 0; i < scan && (int)batch.size() < S->max_batch;) {
                        Req *r = S->queue[i];
                        const double w = work(S, r);
                        if (w > w0 * q || w * q < w0) {
                            ++i;
                            continue;
                        }
                        if (!reserve(S, r)) break;
                        S->queue.erase(S->queue.begin() + (std::ptrdiff_t)i);
                        --scan;
                        r->state = kRunning;
                        batch.push_back(r);
                    }
                }
            }
            if (batch.empty()) break;
            const int si = S->free_streams.front();
            S->free_streams.pop_front();
            Batch B;
            prepare(S, si, batch, B);
            // (requests of a batch are retired together once its event passed)
            S->inflight.push_back(std::move(B));
            S->nbatch += 1;
            S->nbatched += (int64_t)batch.size();
        }
        // the copies and launches happen without the lock: only this thread
        // touches the batches in flight and the copy stream
        lk.unlock();
        pump(S);
        lk.lock();
        if (S->stop && S->queue.empty() && S->inflight.empty()) break;
        if (S->inflight.empty())
            S->cv_work.wait(lk);  // idle: until a submit, a release or stop
        else
            S->cv_work.wait_for(lk, std::chrono::microseconds(20));  // poll the events
    }
}

}  // namespace
}  // namespace sell

namespace sell {
namespace {

// Deliver a completed request (lock held): fill *info; a request with nothing
// left on the device is forgotten, a device result stays until its release.
sell_status collect(sell_server *S, std::unordered_map<uint64_t, Req *>::iterator it, sell_request_info *info) {
    Req *r = it->second;
    if (info) {
        info->t_arrive = r->ta;
        info->t_launch = r->tl;
        info->t_done = r->td;
        info->batch = r->batch;
        info->status = r->status;
    }
    r->collected = true;
    const sell_status st = (sell_status)r->status;
    if (!r->keep_y() || r->status != SELL_OK) {
        S->reqs.erase(it);
        delete r;
    }
    if (st != SELL_OK) return fail(st, "sell_server: the request's batch failed");
    return SELL_OK;
}

}  // namespace
}  // namespace sell

using namespace sell;

extern "C" {

sell_status sell_server_create(const sell_handle *mats, int32_t n, const sell_server_opts *o, sell_server_t *out) {
    if (!mats || n < 1 || !o || !out) return fail(SELL_EINVAL, "sell_server_create: bad arguments");
    if (o->max_batch < 1 || o->max_batch > 4096 || o->streams < 1 || o->streams > 16 || o->size_ratio < 0 ||
        o->max_batch_work < 0)
        return fail(SELL_EINVAL,
                    "sell_server_create: need 1 <= max_batch <= 4096, 1 <= streams <= 16, size_ratio >= 0");
    if (o->reserved != 0) return fail(SELL_EINVAL, "sell_server_create: reserved must be 0");
    sell_server *S = new (std::nothrow) sell_server();
    if (!S) return fail(SELL_ENOMEM, "sell_server_create: host allocation failed");
    int dev = 0;
    (void)cudaGetDevice(&dev);
    S->device = dev;
    for (int32_t i = 0; i < n; ++i) {
        if (!mats[i]) {
            delete S;
            return fail(SELL_EINVAL, "sell_server_create: NULL matrix");
        }
        if (mats[i]->device != dev) {
            delete S;
            return fail(SELL_EINVAL, "sell_server_create: matrices must live on the current device");
        }
        S->mats.push_back(mats[i]);
        S->resident += (int64_t)mats[i]->device_bytes;
    }
    S->budget = o->budget_bytes;
    if (S->resident >= S->budget) {
        delete S;
        return fail(SELL_EINVAL, "sell_server_create: the resident matrices fill the budget");
    }
    S->arena_bytes = (S->budget - S->resident) / 256 * 256;
    S->max_batch = o->max_batch;
    S->nstreams = o->streams;
    S->size_ratio = o->size_ratio;
    S->max_work = o->max_batch_work;
    S->al = current_allocator();
    S->arena_base = static_cast<char *>(S->al.get((size_t)S->arena_bytes, nullptr));
    if (!S->arena_base) {
        delete S;
        return fail(SELL_ENOMEM, "sell_server_create: arena allocation failed");
    }
    S->arena.reset((size_t)S->arena_bytes);
    sell_status st = SELL_OK;
    for (int i = 0; i < S->nstreams && st == SELL_OK; ++i) {
        cudaStream_t s = nullptr;
        if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess)
            st = cuda_fail(cudaGetLastError(), "sell_server_create: stream");
        S->streams.push_back(s);
        for (int p = 0; p < 2 && st == SELL_OK; ++p) {
            cudaEvent_t e = nullptr, rd = nullptr;
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess ||
                cudaEventCreateWithFlags(&rd, cudaEventDisableTiming) != cudaSuccess)
                st = cuda_fail(cudaGetLastError(), "sell_server_create: event");
            S->events.push_back(e);
            S->ready.push_back(rd);
        }
        S->free_streams.push_back(i);
    }
    if (st == SELL_OK && cudaStreamCreateWithFlags(&S->h2d, cudaStreamNonBlocking) != cudaSuccess)
        st = cuda_fail(cudaGetLastError(), "sell_server_create: copy stream");
    if (st == SELL_OK && cudaDeviceSynchronize() != cudaSuccess)
        st = cuda_fail(cudaGetLastError(), "sell_server_create: arena");
    auto destroy_cuda = [](sell_server *T) {
        for (auto s : T->streams)
            if (s) (void)cudaStreamDestroy(s);
        if (T->h2d) (void)cudaStreamDestroy(T->h2d);
        for (auto e : T->events)
            if (e) (void)cudaEventDestroy(e);
        for (auto e : T->ready)
            if (e) (void)cudaEventDestroy(e);
    };
    if (st != SELL_OK) {
        destroy_cuda(S);
        S->al.put(S->arena_base, nullptr);
        delete S;
        return st;
    }
    try {
        S->thr = std::thread(scheduler, S);
    } catch (...) {
        destroy_cuda(S);
        S->al.put(S->arena_base, nullptr);
        delete S;
        return fail(SELL_ENOMEM, "sell_server_create: cannot start the scheduler thread");
    }
    *out = S;
    return SELL_OK;
}

sell_status sell_server_submit(sell_server_t S, int32_t mid, const void *X, int32_t k, void *Y, uint32_t flags,
                               uint64_t *id) {
    if (!S || !id) return fail(SELL_EINVAL, "sell_server_submit: NULL argument");
    if (mid < 0 || mid >= (int32_t)S->mats.size()) return fail(SELL_EINVAL, "sell_server_submit: bad matrix id");
    if (k < 1) return fail(SELL_EINVAL, "sell_server_submit: need k >= 1");
    if (flags & ~(SELL_SPMV_ACCUMULATE | kCompFlags))
        return fail(SELL_EINVAL, "sell_server_submit: unsupported flags");
    const sell_matrix *h = S->mats[mid];
    if ((flags & kCompFlags) && h->store_type == SELL_F64)
        return fail(SELL_EUNSUPPORTED, "compensated accumulation needs F32/BF16 storage");
    if ((flags & SELL_SPMV_ACCUMULATE) && !Y)
        return fail(SELL_EINVAL, "sell_server_submit: accumulating needs a host y");
    if ((h->ncols > 0 && !X) || (X && !is_pinned_host(X)) || (Y && !is_pinned_host(Y)))
        return fail(SELL_EINVAL, "sell_server_submit: X and Y must be page-locked host memory");
    Req *r = new (std::nothrow) Req();
    if (!r) return fail(SELL_ENOMEM, "sell_server_submit: host allocation failed");
    r->mid = mid;
    r->k = k;
    r->flags = flags;
    r->X = X;
    r->Y = Y;
    sizes(S, r);
    if ((int64_t)footprint(r) > S->arena_bytes) {
        delete r;
        return fail(SELL_EINVAL, "sell_server_submit: the request alone exceeds the budget");
    }
    {
        std::lock_guard<std::mutex> g(S->mu);
        if (S->stop) {
            delete r;
            return fail(SELL_EINVAL, "sell_server_submit: the server is stopping");
        }
        r->id = S->next_id++;
        r->ta = now_s();
        S->reqs[r->id] = r;
        S->queue.push_back(r);
        S->nreq += 1;
        *id = r->id;
    }
    S->cv_work.notify_one();
    return SELL_OK;
}

sell_status sell_server_wait(sell_server_t S, uint64_t id, double timeout_s, sell_request_info *info) {
    if (!S) return fail(SELL_EINVAL, "sell_server_wait: NULL server");
    std::unique_lock<std::mutex> lk(S->mu);
    const auto until = std::chrono::steady_clock::now() +
                       std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                           std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 0));
    for (bool timed_out = false;;) {
        // looked up again after every wake-up: while this thread slept, another
        // one may have delivered the request (sell_server_next) or released it,
        // and the request may no longer exist
        auto it = S->reqs.find(id);
        if (it == S->reqs.end())
            return fail(SELL_EINVAL, "sell_server_wait: unknown request (or delivered to another caller)");
        if (it->second->state == kDone) return collect(S, it, info);
        if (timed_out) return fail(SELL_ETIMEOUT, "sell_server_wait: timed out");
        timed_out = S->cv_done.wait_until(lk, until) == std::cv_status::timeout;
    }
}

sell_status sell_server_next(sell_server_t S, double timeout_s, uint64_t *id, sell_request_info *info) {
    if (!S || !id) return fail(SELL_EINVAL, "sell_server_next: NULL argument");
    std::unique_lock<std::mutex> lk(S->mu);
    const auto until = std::chrono::steady_clock::now() +
                       std::chrono::duration_cast<std::chrono::steady_clock::duration>(
                           std::chrono::duration<double>(timeout_s > 0 ? timeout_s : 0));
    for (;;) {
        while (!S->completed.empty()) {
            const uint64_t rid = S->completed.front();
            S->completed.pop_front();
            auto it = S->reqs.find(rid);
            if (it == S->reqs.end() || it->second->collected) continue;  // collected by a wait
            *id = rid;
            return collect(S, it, info);
        }
        if (S->cv_done.wait_until(lk, until) == std::cv_status::timeout && S->completed.empty())
            return fail(SELL_ETIMEOUT, "sell_server_next: no request completed in time");
    }
}

sell_status sell_server_result(sell_server_t S, uint64_t id, void **dev_y) {
    if (!S || !dev_y) return fail(SELL_EINVAL, "sell_server_result: NULL argument");
    std::lock_guard<std::mutex> g(S->mu);
    auto it = S->reqs.find(id);
    if (it == S->reqs.end() || !it->second->keep_y() || it->second->state != kDone)
        return fail(SELL_EINVAL, "sell_server_result: not a completed device-result request");
    *dev_y = S->arena_base + it->second->yoff;
    return SELL_OK;
}

sell_status sell_server_release(sell_server_t S, uint64_t id) {
    if (!S) return fail(SELL_EINVAL, "sell_server_release: NULL server");
    {
        std::lock_guard<std::mutex> g(S->mu);
        auto it = S->reqs.find(id);
        if (it == S->reqs.end() || !it->second->keep_y() || it->second->state != kDone)
            return fail(SELL_EINVAL, "sell_server_release: not a completed device-result request");
        release_y(S, it->second);
        delete it->second;
        S->reqs.erase(it);
    }
    S->cv_work.notify_one();
    return SELL_OK;
}

sell_status sell_server_stats(sell_server_t S, sell_server_stats_t *st) {
    if (!S || !st) return fail(SELL_EINVAL, "sell_server_stats: NULL argument");
    std::lock_guard<std::mutex> g(S->mu);
    st->requests = S->nreq;
    st->batches = S->nbatch;
    st->batched_requests = S->nbatched;
    st->queued = (int64_t)S->queue.size();
    st->resident_bytes = S->resident;
    st->budget_bytes = S->budget;
    st->in_use_bytes = S->resident + S->used;
    st->peak_bytes = S->resident + S->peak_used;
    return SELL_OK;
}

sell_status sell_server_destroy(sell_server_t S) {
    if (!S) return SELL_OK;
    {
        // results still held on the device die with the server; returning
        // them first lets every queued request be admitted and finish
        std::lock_guard<std::mutex> g(S->mu);
        S->stop = true;
        for (auto it = S->reqs.begin(); it != S->reqs.end();) {
            Req *r = it->second;
            if (r->state == kDone && r->keep_y() && r->reserved) {
                release_y(S, r);
                delete r;
                it = S->reqs.erase(it);
            } else {
                ++it;
            }
        }
    }
    S->cv_work.notify_all();
    if (S->thr.joinable()) S->thr.join();
    for (auto s : S->streams) (void)cudaStreamSynchronize(s);
    if (S->h2d) (void)cudaStreamSynchronize(S->h2d);
    for (auto s : S->streams) (void)cudaStreamDestroy(s);
    if (S->h2d) (void)cudaStreamDestroy(S->h2d);
    for (auto e : S->events) (void)cudaEventDestroy(e);
    for (auto e : S->ready) (void)cudaEventDestroy(e);
    for (auto &ce : S->copying) (void)cudaEventDestroy(ce.first);
    for (auto e : S->spare) (void)cudaEventDestroy(e);
    S->al.put(S->arena_base, nullptr);
    (void)cudaDeviceSynchronize();
    for (auto &kv : S->reqs) delete kv.second;
    delete S;
    return SELL_OK;
}

}  // extern "C"
