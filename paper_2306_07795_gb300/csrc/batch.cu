// batch.cu -- many BMMC permutations of different sizes in one persistent
// launch per phase.
//
// A batch binds plans[i] to (ins[i], outs[i]).  Its work is the list of
// thread-block items of every pass: phase 1 holds the first pass of every
// plan (in -> out for one-pass plans, in -> workspace slice for two-pass
// plans), phase 2 the second pass of the two-pass plans (workspace -> out,
// Sec. 5.2).  Each phase is one persistent kernel per element size present:
// a grid of (SMs x resident blocks) thread blocks, each walking a contiguous
// range of items, so that small arrays (the paper notes that arrays under
// 2^20 elements cannot fill a GPU, Sec. 6) share the machine with large ones
// instead of each needing its own launch.  A block reloads a pass's tables
// into shared memory only when its range crosses into the next array.
#include <cuda_runtime.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "bmmc.h"
#include "bmmc_batch.h"
#include "debug_hooks.hpp"
#include "guard.hpp"
#include "plan_internal.hpp"
#include "tile_body.cuh"

using namespace bmmc;

namespace {

// One (array, pass) of a phase.
struct BatchEntry {
    const uint8_t *src;
    uint8_t *dst;
    uint64_t first_item;  // items of the phase before this entry
    uint32_t desc;        // index of the pass's tables in the desc array
    uint32_t pad;
};
static_assert(sizeof(BatchEntry) == 32, "BatchEntry layout");

// Pass tables are stored, and staged in shared memory, in 128-byte slots.
constexpr uint32_t kDescSlot = (uint32_t)((sizeof(PassDesc) + 127) & ~(size_t)127);
constexpr uint32_t kThreads = 256;

// Shared memory: `slots` table slots, then `slots` tile buffers (slots = 3,
// or 2 when three tile buffers do not fit).  A block's items rotate over the
// slots: while one item is gathered and stored from its buffer, the loads of
// the block's next item are already in flight into the next buffer (cp.async
// groups).  With three slots the loads issued for item i + 2 go to the buffer
// item i - 1 used, which every thread finished reading before the barrier of
// item i, so one barrier per item suffices; two slots need a second barrier
// after the stores.  The last 32 bytes record which table each slot holds
// and the chunks a block has claimed ahead.
constexpr uint32_t kMaxSlots = 3;
template <int E_LOG>
__global__ void __launch_bounds__(kThreads, 4)
    bmmc_batch_pass(const BatchEntry *__restrict__ ent, uint32_t count, uint32_t total,
                    const uint8_t *__restrict__ descs, uint32_t tile_bytes, uint32_t slots,
                    uint32_t chunk, uint32_t *__restrict__ ctr)
{
    extern __shared__ __align__(128) uint8_t smem[];
    const uint32_t s0 = (uint32_t)__cvta_generic_to_shared(smem);
    const uint32_t tid = threadIdx.x;

    // The items are cut into chunks of `chunk` consecutive items.  Block b
    // starts with chunk b; the chunks after the first G (G blocks) are
    // claimed from a counter as blocks finish theirs, so a block slowed down
    // by its neighbours takes fewer of them and the launch ends evenly.
    // Blocks running at the same time still take nearby chunks.  ctr[0]
    // counts claims and ctr[1] finished blocks; the last block to finish
    // resets both, so the next launch of the batch starts from zero.
    const uint32_t G = gridDim.x;
    uint32_t cid = blockIdx.x;
    uint32_t cend = 0;
    // Launched with programmatic stream serialization (phase 2 is scheduled
    // while phase 1 drains); nothing above touched global memory.
    dev::grid_dependency_wait();
    dev::allow_dependent_launch();
    // Table held by each slot, in shared memory after the tile buffers.
    // Every thread writes the same value; it is read only after a barrier.
    volatile uint32_t *held =
        reinterpret_cast<volatile uint32_t *>(smem + slots * (kDescSlot + tile_bytes));
    // Chunks claimed ahead: chunk j of this block (j >= 1) is ring[j % 3],
    // written by thread 0 at least one barrier before any thread reads it.
    volatile uint32_t *ring = held + 4;
    if (tid < kMaxSlots) held[tid] = 0xffffffffu;
    if (tid == 0) {
        const uint32_t c0 = atomicAdd(&ctr[0], 2u);
        ring[1] = G + c0;
        ring[2] = G + c0 + 1;
    }
    auto block_done = [&]() {
        if (tid == 0) {
            __threadfence();  // this block's claims come before its count
            if (atomicAdd(&ctr[1], 1u) == G - 1) {
                ctr[0] = 0;
                ctr[1] = 0;
            }
        }
    };
    __syncthreads();
    if ((uint64_t)cid * chunk >= total) {
        block_done();
        return;
    }
    const uint32_t begin = cid * chunk;
    cend = total - begin > chunk ? begin + chunk : total;
    uint32_t seq = 0;             // this block's chunks so far, minus one
    uint32_t pending = 0;         // thread 0: a claim not yet in the ring
    int pending_slot = -1;
    // the item after `it` for this block (total when there is none); moves to
    // the next claimed chunk when `it` ends the current one
    auto advance = [&](uint32_t it) -> uint32_t {
        if (it + 1 < cend) return it + 1;
        ++seq;
        cid = ring[seq % 3];
        if (tid == 0) {  // the chunk after the next two; stored next turn
            pending = atomicAdd(&ctr[0], 1u);
            pending_slot = (int)((seq + 2) % 3);
        }
        const uint64_t start = (uint64_t)cid * chunk;
        if (start >= total) return total;
        cend = total - (uint32_t)start > chunk ? (uint32_t)start + chunk : total;
        return (uint32_t)start;
    };

    // Advance *a to the last entry whose first item is <= item, by doubling
    // steps and then bisection: O(log skipped) dependent loads, one for the
    // next item of the same array.
    auto find = [&](uint32_t item, uint32_t *a) {
        uint32_t lo = *a, step = 1, hi;
        for (;;) {
            const uint32_t probe = lo + step;
            if (probe >= count || ent[probe].first_item > item) {
                hi = (probe < count ? probe : count) - 1;
                break;
            }
            lo = probe;
            step <<= 1;
        }
        while (lo < hi) {
            const uint32_t mid = (lo + hi + 1) >> 1;
            if (ent[mid].first_item <= item) lo = mid;
            else hi = mid - 1;
        }
        *a = lo;
    };
    // Find the entry of `item` and make slot `slot` hold its tables.  The
    // slot's previous user finished before the last barrier.
    auto stage = [&](uint32_t item, int slot, uint32_t *a) {
        find(item, a);
        const uint32_t desc = ent[*a].desc;
        if (desc != held[slot]) {
            const uint4 *src = reinterpret_cast<const uint4 *>(descs + (size_t)desc * kDescSlot);
            uint4 *dst = reinterpret_cast<uint4 *>(smem + slot * kDescSlot);
            for (uint32_t w = tid; w < kDescSlot / 16; w += blockDim.x) dst[w] = src[w];
            __syncthreads();
            held[slot] = desc;
        }
    };
    auto table = [&](int slot) -> const PassDesc & {
        return *reinterpret_cast<const PassDesc *>(smem + slot * kDescSlot);
    };
    auto buffer = [&](int slot) {
        return s0 + slots * kDescSlot + (uint32_t)slot * tile_bytes;
    };
    // Thread part of the addresses of the pass last seen (consecutive items
    // of a block almost always belong to the same pass).
    uint32_t tp_desc = 0xffffffffu;
    dev::TileAddr tp;
    auto addr = [&](const PassDesc &d, uint32_t a, uint32_t item) {
        if (ent[a].desc != tp_desc) {
            tp = dev::thread_part(d);
            tp_desc = ent[a].desc;
        }
        return dev::with_block(d, tp, item - (uint32_t)ent[a].first_item);
    };
    auto issue = [&](uint32_t item, uint32_t a, int slot) {
        const PassDesc &d = table(slot);
        if (!d.naive && tid < (1u << d.thread_bits))
            dev::tile_load<E_LOG>(d, addr(d, a, item), ent[a].src, buffer(slot));
        asm volatile("cp.async.commit_group;\n" ::: "memory");
    };

    uint32_t a_cur = 0;
    stage(begin, 0, &a_cur);
    issue(begin, a_cur, 0);
    int slot = 0;
    for (uint32_t item = begin; item < total;) {
        const int next = slot + 1 == (int)slots ? 0 : slot + 1;
        uint32_t a_next = a_cur;
        if (pending_slot >= 0) {  // thread 0 only; a barrier has passed
            ring[pending_slot] = G + pending;
            pending_slot = -1;
        }
        const uint32_t nxt = advance(item);
        if (nxt < total) {
            stage(nxt, next, &a_next);
            issue(nxt, a_next, next);
            asm volatile("cp.async.wait_group 1;\n" ::: "memory");
        } else {
            asm volatile("cp.async.wait_group 0;\n" ::: "memory");
        }
        __syncthreads();  // every thread's copies of this item have landed
        const PassDesc &d = table(slot);
        if (d.naive) {
            dev::run_naive<E_LOG>(d, ent[a_cur].src, ent[a_cur].dst);
        } else if (tid < (1u << d.thread_bits)) {
            dev::tile_store<E_LOG, dev::kKeyNone>(d, addr(d, a_cur, item), ent[a_cur].dst,
                                                  buffer(slot));
        }
        if (slots == 2) __syncthreads();  // buffer `slot` is free for item + 2
        a_cur = a_next;
        slot = next;
        item = nxt;
    }
    block_done();
}

struct Group {
    int e_log = 0;
    int phase = 0;
    uint32_t count = 0;
    uint64_t total = 0;
    size_t entry_offset = 0;  // byte offset of its entries in the device block
    size_t ctr_offset = 0;    // byte offset of its two chunk counters
    uint32_t smem = 0;
    uint32_t tile_bytes = 0;  // largest tile buffer of the group's passes
    uint32_t slots = 0;       // tile buffers (3, or 2 when 3 do not fit)
    uint32_t chunk = 0;       // consecutive items a block takes at a time
    uint32_t grid = 0;
    uint32_t arrays = 0;
};

template <int E_LOG>
cudaError_t launch_group(const Group &g, uint8_t *dmem, cudaStream_t s)
{
    const BatchEntry *ent = reinterpret_cast<const BatchEntry *>(dmem + g.entry_offset);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(g.grid);
    cfg.blockDim = dim3(kThreads);
    cfg.dynamicSmemBytes = g.smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, bmmc_batch_pass<E_LOG>, ent, g.count, (uint32_t)g.total,
                              static_cast<const uint8_t *>(dmem), g.tile_bytes, g.slots,
                              g.chunk, reinterpret_cast<uint32_t *>(dmem + g.ctr_offset));
}

// Shared memory of a group with `slots` tile buffers.
uint32_t group_smem(uint32_t slots, uint32_t tile_bytes)
{
    return slots * (kDescSlot + tile_bytes) + 32;
}

// Three tile buffers if they fit in a block's shared memory, else two;
// false if not even two fit (tiles of 128 KiB).
bool choose_slots(Group *g, int max_smem)
{
    for (uint32_t slots = kMaxSlots; slots >= 2; --slots) {
        if (group_smem(slots, g->tile_bytes) <= (uint32_t)max_smem) {
            g->slots = slots;
            g->smem = group_smem(slots, g->tile_bytes);
            return true;
        }
    }
    return false;
}

template <int E_LOG>
cudaError_t prepare_group(Group *g, int sms)
{
    cudaError_t err = cudaFuncSetAttribute(bmmc_batch_pass<E_LOG>,
                                           cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)g->smem);
    if (err != cudaSuccess) return err;
    int per_sm = 0;
    err = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, bmmc_batch_pass<E_LOG>,
                                                        kThreads, g->smem);
    if (err != cudaSuccess) return err;
    if (per_sm < 1) per_sm = 1;
    uint64_t grid = (uint64_t)sms * (uint64_t)per_sm;
    if (grid > g->total) grid = g->total;
    g->grid = (uint32_t)grid;
    // Chunks of about 1/64 of a block's share of the items, at least 16: the
    // blocks resident at a time then work on nearby tiles, while a block
    // still reloads tables rarely.  (On 128 arrays of 2^10..2^24 elements
    // this measured 3-5 % faster than one contiguous range per block, and
    // within 1 % of it on 4096 arrays; chunks of 4 items lost 7 % there.)
    const uint64_t per = (g->total + grid - 1) / grid;
    uint64_t chunk = per / 64;
    if (chunk < 16) chunk = 16;
    if (chunk > per) chunk = per;
    g->chunk = (uint32_t)chunk;
    return cudaSuccess;
}

uint64_t round_up(uint64_t v, uint64_t a) { return (v + a - 1) / a * a; }

struct Range {
    uintptr_t lo, hi;
    bool writable;
};

bool ranges_conflict(std::vector<Range> r)
{
    std::sort(r.begin(), r.end(), [](const Range &a, const Range &b) { return a.lo < b.lo; });
    // any overlap involving a writable range is a conflict; read-only ranges
    // may overlap each other (several plans may read one input)
    uintptr_t max_hi_w = 0, max_hi_any = 0;
    for (const Range &x : r) {
        if (x.lo < max_hi_w) return true;                 // overlaps an earlier writable
        if (x.writable && x.lo < max_hi_any) return true;  // writable overlaps anything
        if (x.writable) max_hi_w = std::max(max_hi_w, x.hi);
        max_hi_any = std::max(max_hi_any, x.hi);
    }
    return false;
}

}  // namespace

struct bmmc_batch_s {
    int device = -1;
    uint8_t *dmem = nullptr;  // caller-owned table memory
    std::vector<Group> groups;
    uint64_t bytes_moved = 0;
};

namespace {

// At most one launch group per (phase, element size).
constexpr int kMaxGroups = 6;
constexpr size_t kCounterBytes = 16;  // per group: claims, finished blocks

// Bytes of the device tables of a batch: one 128-byte slot per pass, then
// one BatchEntry per (array, pass), then the chunk counters of each group.
size_t table_bytes(const bmmc_plan *plans, int count)
{
    size_t passes = 0;
    for (int i = 0; i < count; ++i)
        if (plans[i]) passes += (size_t)plans[i]->npass;
    return passes * kDescSlot + passes * sizeof(BatchEntry) + kMaxGroups * kCounterBytes;
}

int batch_create_impl(bmmc_batch *out, const bmmc_plan *plans, int count,
                      const void *const *ins, void *const *outs, void *ws, void *table,
                      bmmc_stream_t stream);
int batch_describe_impl(bmmc_batch b, char *buf, size_t len);

}  // namespace

extern "C" {

size_t bmmc_batch_workspace_bytes(const bmmc_plan *plans, int count)
{
    if (!plans || count <= 0) return 0;
    uint64_t total = 0;
    for (int i = 0; i < count; ++i)
        if (plans[i] && plans[i]->npass == 2) total = round_up(total, 256) + plans[i]->bytes();
    return (size_t)total;
}

size_t bmmc_batch_table_bytes(const bmmc_plan *plans, int count)
{
    if (!plans || count <= 0) return 0;
    return table_bytes(plans, count);
}

int bmmc_batch_create(bmmc_batch *out, const bmmc_plan *plans, int count,
                      const void *const *ins, void *const *outs, void *ws, void *table,
                      bmmc_stream_t stream)
{
    return guarded(
        [&] { return batch_create_impl(out, plans, count, ins, outs, ws, table, stream); });
}

int bmmc_batch_execute(bmmc_batch b, bmmc_stream_t stream)
{
    if (!b) return BMMC_ERR_INVALID;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev != b->device) return BMMC_ERR_INVALID;
    for (const Group &g : b->groups) {
        if (debug_fail_launch()) return BMMC_ERR_CUDA;
        cudaError_t err;
        switch (g.e_log) {
        case 2: err = launch_group<2>(g, b->dmem, (cudaStream_t)stream); break;
        case 3: err = launch_group<3>(g, b->dmem, (cudaStream_t)stream); break;
        default: err = launch_group<4>(g, b->dmem, (cudaStream_t)stream); break;
        }
        if (err != cudaSuccess) return BMMC_ERR_CUDA;
    }
    return BMMC_OK;
}

int bmmc_batch_num_launches(bmmc_batch b) { return b ? (int)b->groups.size() : BMMC_ERR_INVALID; }

int bmmc_batch_describe(bmmc_batch b, char *buf, size_t len)
{
    return guarded([&] { return batch_describe_impl(b, buf, len); });
}

void bmmc_batch_destroy(bmmc_batch b)
{
    delete b;  // the table memory belongs to the caller
}

int bmmc_execute_batch(const bmmc_plan *plans, const void *const *ins, void *const *outs,
                       int count, bmmc_stream_t stream)
{
    if (!plans || !ins || !outs || count <= 0) return BMMC_ERR_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    const size_t ws_bytes = bmmc_batch_workspace_bytes(plans, count);
    const size_t tab_bytes = bmmc_batch_table_bytes(plans, count);
    if (!tab_bytes) return BMMC_ERR_INVALID;
    void *table = nullptr, *ws = nullptr;
    if (debug_fail_alloc()) return BMMC_ERR_OOM;
    if (cudaMallocAsync(&table, tab_bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return BMMC_ERR_OOM;
    }
    if (ws_bytes && cudaMallocAsync(&ws, ws_bytes, s) != cudaSuccess) {
        cudaGetLastError();
        cudaFreeAsync(table, s);
        return BMMC_ERR_OOM;
    }
    bmmc_batch b = nullptr;
    int rc = bmmc_batch_create(&b, plans, count, ins, outs, ws, table, stream);
    if (rc == BMMC_OK) rc = bmmc_batch_execute(b, stream);
    bmmc_batch_destroy(b);
    // stream order frees the memory after the launches
    if (ws) cudaFreeAsync(ws, s);
    cudaFreeAsync(table, s);
    return rc;
}

}  // extern "C"

namespace {

int batch_create_impl(bmmc_batch *out, const bmmc_plan *plans, int count,
                      const void *const *ins, void *const *outs, void *ws, void *table,
                      bmmc_stream_t stream)
{
    if (!out) return BMMC_ERR_INVALID;
    *out = nullptr;
    if (!plans || !ins || !outs || count <= 0 || !table) return BMMC_ERR_INVALID;
    if ((uintptr_t)table & 15u) return BMMC_ERR_ALIGN;
    const size_t ws_need = bmmc_batch_workspace_bytes(plans, count);
    if (ws_need && !ws) return BMMC_ERR_INVALID;
    if ((uintptr_t)ws & 15u) return BMMC_ERR_ALIGN;

    // Workspace slices and overlap checks.
    std::vector<uint8_t *> slice(count, nullptr);
    std::vector<Range> ranges;
    ranges.reserve(3 * (size_t)count);
    uint64_t off = 0;
    for (int i = 0; i < count; ++i) {
        const bmmc_plan p = plans[i];
        if (!p || !ins[i] || !outs[i] || p->derived < p->npass) return BMMC_ERR_INVALID;
        if (((uintptr_t)ins[i] | (uintptr_t)outs[i]) & 15u) return BMMC_ERR_ALIGN;
        const uint64_t b = p->bytes();
        ranges.push_back({(uintptr_t)ins[i], (uintptr_t)ins[i] + b, false});
        ranges.push_back({(uintptr_t)outs[i], (uintptr_t)outs[i] + b, true});
        if (p->npass == 2) {
            off = round_up(off, 256);
            slice[i] = (uint8_t *)ws + off;
            ranges.push_back({(uintptr_t)slice[i], (uintptr_t)slice[i] + b, true});
            off += b;
        }
    }
    if (ranges_conflict(ranges)) return BMMC_ERR_ALIAS;

    // Pass tables: one slot per (plan, pass).
    std::vector<uint32_t> desc0(count), desc1(count);
    uint32_t ndesc = 0;
    for (int i = 0; i < count; ++i) {
        desc0[i] = ndesc++;
        if (plans[i]->npass == 2) desc1[i] = ndesc++;
    }
    // Groups in launch order: phase 1 then phase 2, element sizes 4, 8, 16.
    std::vector<Group> groups;
    std::vector<BatchEntry> entries;
    uint64_t moved = 0;
    for (int phase = 0; phase < 2; ++phase) {
        for (int e_log = 2; e_log <= 4; ++e_log) {
            Group g;
            g.e_log = e_log;
            g.phase = phase;
            g.entry_offset = entries.size() * sizeof(BatchEntry);
            uint32_t max_smem = 0;
            for (int i = 0; i < count; ++i) {
                const bmmc_plan p = plans[i];
                if (p->e_log != e_log || phase >= p->npass) continue;
                const PassDesc &d = p->desc[phase];
                BatchEntry en;
                memset(&en, 0, sizeof(en));
                if (p->npass == 1) {
                    en.src = (const uint8_t *)ins[i];
                    en.dst = (uint8_t *)outs[i];
                } else if (phase == 0) {
                    en.src = (const uint8_t *)ins[i];
                    en.dst = slice[i];
                } else {
                    en.src = slice[i];
                    en.dst = (uint8_t *)outs[i];
                }
                en.first_item = g.total;
                en.desc = phase == 0 ? desc0[i] : desc1[i];
                entries.push_back(en);
                g.total += d.naive ? 1ull : (1ull << d.n_cta);
                g.count += 1;
                if (!d.naive) max_smem = std::max(max_smem, d.smem_bytes);
                moved += 2 * p->bytes();
            }
            if (g.count == 0) {
                entries.resize(g.entry_offset / sizeof(BatchEntry));
                continue;
            }
            // the kernel counts items in 32 bits (2^32 items of >= 512 bytes
            // would exceed any device memory)
            if (g.total > 0xffffffffull) return BMMC_ERR_TOO_LARGE;
            g.arrays = g.count;
            g.tile_bytes = (max_smem + 127u) & ~127u;
            g.slots = kMaxSlots;
            g.smem = group_smem(g.slots, g.tile_bytes);
            groups.push_back(g);
        }
    }

    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return BMMC_ERR_CUDA;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return BMMC_ERR_CUDA;
    int max_smem = 0;
    if (cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) !=
        cudaSuccess)
        return BMMC_ERR_CUDA;
    for (Group &g : groups) {
        if (!choose_slots(&g, max_smem)) return BMMC_ERR_UNSUPPORTED;
        cudaError_t err = cudaSuccess;
        switch (g.e_log) {
        case 2: err = prepare_group<2>(&g, sms); break;
        case 3: err = prepare_group<3>(&g, sms); break;
        default: err = prepare_group<4>(&g, sms); break;
        }
        if (err != cudaSuccess) {
            cudaGetLastError();
            return BMMC_ERR_CUDA;
        }
    }

    // One device block: pass tables, then the entries of every group.
    const size_t desc_bytes = (size_t)ndesc * kDescSlot;
    const size_t ent_bytes = entries.size() * sizeof(BatchEntry);
    // the counters start at zero (uploaded with the tables)
    std::vector<uint8_t> host(desc_bytes + ent_bytes + groups.size() * kCounterBytes, 0);
    for (int i = 0; i < count; ++i) {
        memcpy(host.data() + (size_t)desc0[i] * kDescSlot, &plans[i]->desc[0], sizeof(PassDesc));
        if (plans[i]->npass == 2)
            memcpy(host.data() + (size_t)desc1[i] * kDescSlot, &plans[i]->desc[1],
                   sizeof(PassDesc));
    }
    memcpy(host.data() + desc_bytes, entries.data(), ent_bytes);
    for (size_t gi = 0; gi < groups.size(); ++gi) {
        groups[gi].entry_offset += desc_bytes;
        groups[gi].ctr_offset = desc_bytes + ent_bytes + gi * kCounterBytes;
    }

    bmmc_batch_s *b = new (std::nothrow) bmmc_batch_s();
    if (!b) return BMMC_ERR_OOM;
    b->dmem = (uint8_t *)table;
    // From pageable memory the copy is staged before the call returns, so the
    // host vector may go; the device side is ordered on `stream`.
    if (cudaMemcpyAsync(b->dmem, host.data(), host.size(), cudaMemcpyHostToDevice,
                        (cudaStream_t)stream) != cudaSuccess) {
        cudaGetLastError();
        delete b;
        return BMMC_ERR_CUDA;
    }
    b->device = dev;
    b->groups = groups;
    b->bytes_moved = moved;
    *out = b;
    return BMMC_OK;
}

int batch_describe_impl(bmmc_batch b, char *buf, size_t len)
{
    if (!b) return BMMC_ERR_INVALID;
    std::string s = "{\"launches\": [";
    for (size_t i = 0; i < b->groups.size(); ++i) {
        const Group &g = b->groups[i];
        char tmp[256];
        snprintf(tmp, sizeof(tmp),
                 "%s{\"phase\": %d, \"elem_bytes\": %d, \"arrays\": %u, \"items\": %llu, "
                 "\"grid\": %u, \"chunk\": %u, \"threads\": %u, \"smem_bytes\": %u}",
                 i ? ", " : "", g.phase + 1, 1 << g.e_log, g.arrays,
                 (unsigned long long)g.total, g.grid, g.chunk, kThreads, g.smem);
        s += tmp;
    }
    char tail[64];
    snprintf(tail, sizeof(tail), "], \"bytes_moved\": %llu}", (unsigned long long)b->bytes_moved);
    s += tail;
    if (buf && len) {
        size_t cpy = s.size() < len - 1 ? s.size() : len - 1;
        memcpy(buf, s.data(), cpy);
        buf[cpy] = 0;
    }
    return (int)s.size();
}

}  // namespace
