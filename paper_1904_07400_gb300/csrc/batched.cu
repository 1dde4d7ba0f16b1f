// Many independent force solves (grids of any size and order) in ONE persistent launch.
//
// Work list: every row-transform item (a group of TR rows of one grid), then every column
// item (one frequency column of one grid), then every inverse-row item (a group of TR rows
// of one force component of one grid).  Blocks take items in list order from an atomic
// ticket.  A column item of grid d waits until all row items of grid d are finished, an
// inverse-row item until all column items of d are; since items are taken in order, every
// item a waiting block depends on is already held by a running block, so the waits end.
// Each wait is bounded (about a second); a wait that runs out sets the batch's error word
// to TDG_ERR_TIMEOUT, skips its item and lets the launch finish.
//
// The item bodies are the generic passes (generic_passes.cuh), so any grid whose padded
// periods are 2^a 3^b works; the batch's dynamic shared memory is the largest any item
// needs.
#include <cuda_runtime.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "generic_passes.cuh"
#include "tdg_internal.cuh"

namespace tdg {
namespace {

struct BatchDisk {
    const float* sigma;
    float* fx;
    float* fy;
    cpx<float>* z;
    cpx<float>* gx;
    cpx<float>* gy;
    const cpx<float>* twx;
    const cpx<float>* twy;
    const float* spec;
    FftPlan rows;  // length P_y / 2 complex transform
    FftPlan cols;  // length P_x complex transform
    Tiled tiled;
    int nx, ny, hy, solve;
    int nA, nB, nC;  // items per pass
};

constexpr int kPhases = 3;
constexpr long long kSpinLimit = 1000000;  // ~1 s with 1 us naps

struct BatchDev {
    const BatchDisk* disks;
    const int* start;   // [3][count + 1] prefix sums of items per pass
    int* done;          // [3][count] finished items per pass and grid
    int* ticket;
    int* err;
    int count;
    int total;
    int withhold;       // grid whose row-pass completions are not counted (test hook), or -1
};

__device__ int find_disk(const int* pref, int count, int item) {
    int lo = 0, hi = count;  // pref[lo] <= item < pref[hi]
    while (hi - lo > 1) {
        int mid = (lo + hi) / 2;
        if (pref[mid] <= item) lo = mid;
        else hi = mid;
    }
    return lo;
}

constexpr int kBatchEPT = 8;  // values per thread in the batched kernel's transform stages

// one out-of-line function per item kind: each gets its own register allocation instead of
// the union of all three
__device__ __noinline__ void item_rows(const BatchDisk& g, int idx, unsigned char* smem) {
    row_r2c_body<float, kBatchEPT>(g.sigma, g.nx, g.ny, g.ny, g.solve, g.rows, g.twy, g.z, g.tiled, g.hy, idx, smem);
}

__device__ __noinline__ void item_cols(const BatchDisk& g, int idx, unsigned char* smem) {
    col_conv_body<float, true, kBatchEPT>(g.z, g.tiled, g.nx, g.hy, g.solve, g.cols, g.twx, g.spec, g.gx, g.gy, idx,
                                          smem);
}

__device__ __noinline__ void item_inv(const BatchDisk& g, int idx, unsigned char* smem) {
    const int groups = (g.nx + RowCfg<float>::TR - 1) / RowCfg<float>::TR;
    row_c2r_body<float, kBatchEPT>(g.gx, g.gy, g.tiled, g.nx, g.hy, 0, g.rows, g.twy, g.fx, g.fy, g.ny, idx % groups,
                                   idx / groups, smem);
}

__global__ void __launch_bounds__(512) k_batched(BatchDev b) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int s_item, s_ok;
    const int* startA = b.start;
    const int* startB = b.start + (b.count + 1);
    const int* startC = b.start + 2 * (b.count + 1);
    const int totA = startA[b.count], totB = startB[b.count];
    for (;;) {
        if (threadIdx.x == 0) s_item = atomicAdd(b.ticket, 1);
        __syncthreads();
        const int item = s_item;
        if (item >= b.total) break;
        int phase, local;
        const int* pref;
        if (item < totA) {
            phase = 0;
            local = item;
            pref = startA;
        } else if (item < totA + totB) {
            phase = 1;
            local = item - totA;
            pref = startB;
        } else {
            phase = 2;
            local = item - totA - totB;
            pref = startC;
        }
        const int d = find_disk(pref, b.count, local);
        const int idx = local - pref[d];
        const BatchDisk& g = b.disks[d];
        // wait for this grid's previous pass
        if (threadIdx.x == 0) {
            int ok = 1;
            if (phase > 0) {
                const int need = phase == 1 ? g.nA : g.nB;
                volatile int* cnt = b.done + (phase - 1) * b.count + d;
                long long spins = 0;
                volatile int* errw = b.err;
                while (*cnt < need) {
                    if (++spins > kSpinLimit || *errw != 0) {
                        ok = 0;
                        atomicExch(b.err, (int)TDG_ERR_TIMEOUT);
                        break;
                    }
                    __nanosleep(1000);
                }
                __threadfence();
            }
            s_ok = ok;
        }
        __syncthreads();
        if (s_ok) {
            if (phase == 0)
                item_rows(g, idx, smem_raw);
            else if (phase == 1)
                item_cols(g, idx, smem_raw);
            else
                item_inv(g, idx, smem_raw);
        }
        __syncthreads();
        if (threadIdx.x == 0) {
            __threadfence();
            if (!(phase == 0 && d == b.withhold)) atomicAdd(b.done + phase * b.count + d, 1);
        }
    }
}

}  // namespace
}  // namespace tdg

using namespace tdg;

struct tdg_batch_s {
    int device;
    int count;
    int threads;
    int radix_pref;
    size_t smem;
    int total;
    int blocks;
    std::vector<tdg_plan> plans;
    std::vector<BatchDisk> host;
    BatchDisk* disks;
    int* start;
    int* done;  // done[3][count] then the ticket
    int* err;
    void* work;
    int withhold;
    // per-grid pointers (the streams form launches each grid's own forward path)
    std::vector<const float*> sig;
    std::vector<float*> fxs, fys;
    std::vector<void*> wptr;
    // streams form: 0 = the persistent kernel; n > 0 = grids on n internal streams
    int nstreams;
    std::vector<cudaStream_t> streams;
    std::vector<cudaEvent_t> joins;
    cudaEvent_t fork;
    std::vector<int> lane;  // internal stream of each grid (LPT on the solve cost)
    std::vector<int> order; // grids by decreasing cost
    // persistent kernel on the transform network's item bodies (threads == 64)
    bool net_ok;            // every grid on the network path with sides up to 1024 cells
    NetDisk* ndisks;
    int* nstart;
    int ntotal;
    int nblocks;
    int net_units;          // units per item of the network form
};

namespace {

bool smooth_radices(int L, int pref, FftPlan& fp) {
    fp.L = L;
    fp.nst = 0;
    int e2 = 0, e3 = 0, t = L;
    while (t % 2 == 0) { t /= 2; ++e2; }
    while (t % 3 == 0) { t /= 3; ++e3; }
    if (t != 1) return false;
    for (int i = 0; i < e3; ++i) fp.radix[fp.nst++] = 3;
    if (pref == 1) {
        while (e2 >= 2) { fp.radix[fp.nst++] = 4; e2 -= 2; }
    } else {
        while (e2 >= 3) { fp.radix[fp.nst++] = 8; e2 -= 3; }
        if (e2 == 2) { fp.radix[fp.nst++] = 4; e2 = 0; }
    }
    if (e2 == 1) fp.radix[fp.nst++] = 2;
    return fp.nst <= kMaxStages;
}

size_t row_bytes(int M, int ncols, int solve) {
    const int TR = RowCfg<float>::TR;
    return (size_t)(M + 1) * TR * sizeof(cpx<float>) + (solve ? (size_t)ncols * TR * sizeof(float) : 0) +
           kSolveTab * sizeof(float);
}

tdg_status batch_configure(tdg_batch_s* b) {
    size_t smem = 0;
    int total = 0;
    std::vector<int> start(kPhases * (b->count + 1), 0);
    for (int d = 0; d < b->count; ++d) {
        const Plan& p = tdg_plan_internal(b->plans[d]);
        BatchDisk& g = b->host[d];
        if (!smooth_radices(p.ay.P / 2, b->radix_pref, g.rows) || !smooth_radices(p.ax.P, b->radix_pref, g.cols))
            return TDG_ERR_UNSUPPORTED;
        const int M = p.ay.P / 2;
        smem = std::max(smem, row_bytes(M, p.ny, solve_order(p)));
        smem = std::max(smem, (size_t)p.ax.P * sizeof(cpx<float>) + kSolveTab * sizeof(float));
        // every pass must be covered by the block: the stages hold kEPT values per thread
        if ((long)RowCfg<float>::TR * M > (long)kBatchEPT * b->threads || p.ax.P > kBatchEPT * b->threads)
            return TDG_ERR_UNSUPPORTED;
        const int groups = (p.nx + RowCfg<float>::TR - 1) / RowCfg<float>::TR;
        g.nA = groups;
        g.nB = p.hy;
        g.nC = 2 * groups;
        start[0 * (b->count + 1) + d + 1] = start[0 * (b->count + 1) + d] + g.nA;
        start[1 * (b->count + 1) + d + 1] = start[1 * (b->count + 1) + d] + g.nB;
        start[2 * (b->count + 1) + d + 1] = start[2 * (b->count + 1) + d] + g.nC;
    }
    for (int ph = 0; ph < kPhases; ++ph) total += start[ph * (b->count + 1) + b->count];
    if (smem > 227 * 1024) return TDG_ERR_UNSUPPORTED;
    cudaError_t e = cudaMemcpy(b->disks, b->host.data(), b->count * sizeof(BatchDisk), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->start, start.data(), start.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_batched, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return TDG_ERR_CUDA;
    int per_sm = 0, sms = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_batched, b->threads, smem);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, b->device);
    if (e != cudaSuccess || per_sm < 1) return TDG_ERR_UNSUPPORTED;
    b->smem = smem;
    b->total = total;
    b->blocks = per_sm * sms;  // every block resident: one persistent wave
    return TDG_OK;
}

void streams_free(tdg_batch_s* b) {
    for (cudaStream_t st : b->streams) cudaStreamDestroy(st);
    for (cudaEvent_t ev : b->joins) cudaEventDestroy(ev);
    if (b->fork) cudaEventDestroy(b->fork);
    b->streams.clear();
    b->joins.clear();
    b->fork = nullptr;
    b->nstreams = 0;
}

// relative cost of one grid's solve: nx ny log2(P_x P_y)
double solve_cost(const Plan& p) { return (double)p.nx * p.ny * std::log2((double)p.ax.P * p.ay.P); }

// descriptors of the network persistent form, grids in decreasing cost (largest first, so
// the long items start early and the tail is short); false if a grid is not eligible
tdg_status net_configure(tdg_batch_s* b) {
    b->net_ok = false;
    std::vector<int> ord(b->count);
    std::vector<double> cost(b->count);
    for (int d = 0; d < b->count; ++d) {
        const Plan& p = tdg_plan_internal(b->plans[d]);
        if (!net_batch_units(p, 0)) return TDG_OK;
        cost[d] = solve_cost(p);
        ord[d] = d;
    }
    std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return cost[x] > cost[y]; });
    std::vector<NetDisk> host(b->count);
    // [3][count + 1] prefix sums of items per pass, then [3][count] the grids in each pass's
    // order; both indexed by pass-local position
    std::vector<int> start(kPhases * (b->count + 1) + kPhases * b->count, 0);
    for (int i = 0; i < b->count; ++i) {
        const int d = ord[i];
        const Plan& p = tdg_plan_internal(b->plans[d]);
        NetDisk& g = host[i];
        memset(&g, 0, sizeof(g));
        g.sigma = b->sig[d];
        g.fx = b->fxs[d];
        g.fy = b->fys[d];
        const size_t n_el = (size_t)((p.hy + 1) / 2) * p.nx * 2;  // two-column tiles of Z, G_x, G_y
        g.z = b->wptr[d];
        g.gx = reinterpret_cast<cpx<float>*>(g.z) + n_el;
        g.gy = reinterpret_cast<cpx<float>*>(g.gx) + n_el;
        g.nbx = p.net_tw;
        g.nby = reinterpret_cast<const cpx<float>*>(p.net_tw) + p.ax.P / 2 / 8;
        g.twx = p.tw_x;
        g.twy = p.tw_y;
        g.spec = p.spec_half;
        g.nx = p.nx;
        g.ny = p.ny;
        g.hy = p.hy;
        g.ord = solve_order(p);
        g.lx = p.ax.P / 2;
        g.ly = p.ay.P / 2;
        g.uA = net_batch_units(p, 0);
        g.uB = net_batch_units(p, 1);
        g.uC = net_batch_units(p, 2);
        const int U = b->net_units;
        g.nA = (g.uA + U - 1) / U;
        g.nB = (g.uB + U - 1) / U;
        g.nC = (g.uC + U - 1) / U;
    }
    // each pass hands out its grids grouped by the length of the lines it transforms (rows:
    // ly, columns: lx), longest first and by cost within a group, so that the blocks on an
    // SM mostly run the same item body
    for (int ph = 0; ph < kPhases; ++ph) {
        std::vector<int> po(b->count);
        for (int i = 0; i < b->count; ++i) po[i] = i;
        std::stable_sort(po.begin(), po.end(), [&](int x, int y) {
            const int lx = ph == 1 ? host[x].lx : host[x].ly, ly = ph == 1 ? host[y].lx : host[y].ly;
            return lx > ly;
        });
        int* pref = start.data() + ph * (b->count + 1);
        int* order = start.data() + kPhases * (b->count + 1) + ph * b->count;
        for (int i = 0; i < b->count; ++i) {
            const NetDisk& g = host[po[i]];
            order[i] = po[i];
            pref[i + 1] = pref[i] + (ph == 0 ? g.nA : (ph == 1 ? g.nB : g.nC));
        }
    }
    int total = 0;
    for (int ph = 0; ph < kPhases; ++ph) total += start[ph * (b->count + 1) + b->count];
    cudaError_t e = cudaMemcpy(b->ndisks, host.data(), b->count * sizeof(NetDisk), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(b->nstart, start.data(), start.size() * sizeof(int), cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = net_batch_blocks(b->device, &b->nblocks);
    if (e != cudaSuccess) return TDG_ERR_CUDA;
    b->ntotal = total;
    b->net_ok = true;
    return TDG_OK;
}

void batch_free(tdg_batch_s* b) {
    streams_free(b);
    cudaFree(b->ndisks);
    cudaFree(b->nstart);
    cudaFree(b->disks);
    cudaFree(b->start);
    cudaFree(b->done);
    cudaFree(b->err);
    cudaFree(b->work);
}

}  // namespace

extern "C" {

tdg_status tdg_batch_create(tdg_batch* out, const tdg_plan* plans, int count, const void* const* sigma,
                            void* const* fx, void* const* fy) {
    if (!out || !plans || count < 1 || !sigma || !fx || !fy) return TDG_ERR_INVALID_ARG;
    *out = nullptr;
    for (int d = 0; d < count; ++d) {
        if (!plans[d] || !sigma[d] || !fx[d] || !fy[d]) return TDG_ERR_INVALID_ARG;
        if ((((uintptr_t)sigma[d]) | ((uintptr_t)fx[d]) | ((uintptr_t)fy[d])) & 15u) return TDG_ERR_INVALID_ARG;
        const Plan& p = tdg_plan_internal(plans[d]);
        if (!p.built) return TDG_ERR_NOT_BUILT;
        if (p.prec != TDG_FP32) return TDG_ERR_UNSUPPORTED;
        if (p.device != tdg_plan_internal(plans[0]).device) return TDG_ERR_INVALID_ARG;
    }
    tdg_batch_s* b = new (std::nothrow) tdg_batch_s();
    if (!b) return TDG_ERR_OOM;
    b->device = tdg_plan_internal(plans[0]).device;
    b->count = count;
    b->threads = 512;
    b->radix_pref = 0;
    b->withhold = -1;
    b->nstreams = 0;
    b->fork = nullptr;
    b->net_units = 2;
    b->plans.assign(plans, plans + count);
    b->host.resize(count);
    b->sig.resize(count);
    b->fxs.resize(count);
    b->fys.resize(count);
    b->wptr.resize(count);
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    size_t work = 0;
    std::vector<size_t> off(count);
    for (int d = 0; d < count; ++d) {
        off[d] = work;
        work += (workspace_bytes(tdg_plan_internal(plans[d])) + 255) & ~(size_t)255;
    }
    cudaError_t e = cudaMalloc(&b->work, work);
    if (e == cudaSuccess) e = cudaMalloc(&b->disks, count * sizeof(BatchDisk));
    if (e == cudaSuccess) e = cudaMalloc(&b->start, kPhases * (count + 1) * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->done, (kPhases * count + 1) * sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->err, sizeof(int));
    if (e == cudaSuccess) e = cudaMemset(b->err, 0, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc(&b->ndisks, count * sizeof(NetDisk));
    if (e == cudaSuccess) e = cudaMalloc(&b->nstart, (kPhases * (count + 1) + kPhases * count) * sizeof(int));
    if (e != cudaSuccess) {
        batch_free(b);
        delete b;
        if (prev >= 0) cudaSetDevice(prev);
        return e == cudaErrorMemoryAllocation ? TDG_ERR_OOM : TDG_ERR_CUDA;
    }
    for (int d = 0; d < count; ++d) {
        const Plan& p = tdg_plan_internal(plans[d]);
        BatchDisk& g = b->host[d];
        memset(&g, 0, sizeof(g));
        g.sigma = (const float*)sigma[d];
        g.fx = (float*)fx[d];
        g.fy = (float*)fy[d];
        b->sig[d] = g.sigma;
        b->fxs[d] = g.fx;
        b->fys[d] = g.fy;
        b->wptr[d] = (char*)b->work + off[d];
        g.tiled.tw = RowCfg<float>::TW;
        g.tiled.slab = (size_t)p.nx * g.tiled.tw;
        const size_t n_el = (size_t)p.ntile * g.tiled.slab;
        g.z = reinterpret_cast<cpx<float>*>((char*)b->work + off[d]);
        g.gx = g.z + n_el;
        g.gy = g.gx + n_el;
        g.twx = reinterpret_cast<const cpx<float>*>(p.tw_x);
        g.twy = reinterpret_cast<const cpx<float>*>(p.tw_y);
        g.spec = reinterpret_cast<const float*>(p.spec);
        g.nx = p.nx;
        g.ny = p.ny;
        g.hy = p.hy;
        g.solve = solve_order(p);
    }
    tdg_status st = net_configure(b);
    if (st == TDG_OK) {
        st = batch_configure(b);
        // grids the generic kernel cannot hold may still run on the network form
        if (st == TDG_ERR_UNSUPPORTED && b->net_ok) {
            b->threads = 64;
            st = TDG_OK;
        }
    }
    if (prev >= 0) cudaSetDevice(prev);
    if (st != TDG_OK) {
        batch_free(b);
        delete b;
        return st;
    }
    *out = b;
    return TDG_OK;
}

tdg_status tdg_batch_set_config(tdg_batch b, int threads, int radix_pref) {
    if (!b || (threads != 64 && threads != 256 && threads != 512)) return TDG_ERR_INVALID_ARG;
    if (threads == 64) {  // the persistent kernel on the network's item bodies; radix_pref: units per item
        const int u = radix_pref;
        if (u != 1 && u != 2 && u != 4 && u != 8 && u != 16 && u != 32) return TDG_ERR_INVALID_ARG;
        if (!b->net_ok) return TDG_ERR_UNSUPPORTED;
        int prev = -1;
        cudaGetDevice(&prev);
        cudaSetDevice(b->device);
        const int old_u = b->net_units;
        b->net_units = u;
        tdg_status st = net_configure(b);
        if (st != TDG_OK || !b->net_ok) {
            b->net_units = old_u;
            net_configure(b);
            if (st == TDG_OK) st = TDG_ERR_UNSUPPORTED;
        } else {
            b->threads = 64;
            b->radix_pref = u;
        }
        if (prev >= 0) cudaSetDevice(prev);
        return st;
    }
    if (radix_pref < 0 || radix_pref > 1) return TDG_ERR_INVALID_ARG;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    int old_t = b->threads, old_r = b->radix_pref;
    b->threads = threads;
    b->radix_pref = radix_pref;
    tdg_status st = batch_configure(b);
    if (st != TDG_OK) {
        b->threads = old_t;
        b->radix_pref = old_r;
        batch_configure(b);
    }
    if (prev >= 0) cudaSetDevice(prev);
    return st;
}

tdg_status tdg_batch_set_streams(tdg_batch b, int nstreams) {
    if (!b || nstreams < 0 || nstreams > 32) return TDG_ERR_INVALID_ARG;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    streams_free(b);
    cudaError_t e = cudaSuccess;
    if (nstreams > 0) {
        e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
        for (int k = 0; k < nstreams && e == cudaSuccess; ++k) {
            cudaStream_t st = nullptr;
            cudaEvent_t ev = nullptr;
            e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
            if (e == cudaSuccess) b->streams.push_back(st);
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
            if (e == cudaSuccess) b->joins.push_back(ev);
        }
        if (e == cudaSuccess) {
            // grids by decreasing cost, each to the least-loaded stream
            std::vector<double> cost(b->count), load(nstreams, 0.0);
            b->order.resize(b->count);
            b->lane.assign(b->count, 0);
            for (int d = 0; d < b->count; ++d) {
                cost[d] = solve_cost(tdg_plan_internal(b->plans[d]));
                b->order[d] = d;
            }
            std::stable_sort(b->order.begin(), b->order.end(), [&](int x, int y) { return cost[x] > cost[y]; });
            for (int d : b->order) {
                const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
                b->lane[d] = k;
                load[k] += cost[d];
            }
            b->nstreams = nstreams;
        } else {
            streams_free(b);
        }
    }
    if (prev >= 0) cudaSetDevice(prev);
    return e == cudaSuccess ? TDG_OK : TDG_ERR_CUDA;
}

tdg_status tdg_batch_launch(tdg_batch b, tdg_stream stream) {
    if (!b) return TDG_ERR_INVALID_ARG;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (b->nstreams > 0) {
        // fork onto the internal streams, each grid's own forward path, join back
        cudaError_t e = cudaEventRecord(b->fork, s);
        for (int k = 0; k < b->nstreams && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->streams[k], b->fork, 0);
        for (int i = 0; i < b->count && e == cudaSuccess; ++i) {
            const int d = b->order[i];
            e = launch_forward<float>(tdg_plan_internal(b->plans[d]), b->sig[d], b->fxs[d], b->fys[d], b->wptr[d],
                                      b->streams[b->lane[d]]);
        }
        for (int k = 0; k < b->nstreams && e == cudaSuccess; ++k) {
            e = cudaEventRecord(b->joins[k], b->streams[k]);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(s, b->joins[k], 0);
        }
        if (prev >= 0) cudaSetDevice(prev);
        return e == cudaSuccess ? TDG_OK : TDG_ERR_CUDA;
    }
    cudaError_t e = cudaMemsetAsync(b->done, 0, (kPhases * b->count + 1) * sizeof(int), s);
    if (e == cudaSuccess && b->threads == 64) {
        NetBatchDev dv;
        dv.disks = b->ndisks;
        dv.start = b->nstart;
        dv.done = b->done;
        dv.ticket = b->done + kPhases * b->count;
        dv.err = b->err;
        dv.count = b->count;
        dv.total = b->ntotal;
        dv.units = b->net_units;
        // the test hook names a grid in creation order; the network form orders by cost
        dv.withhold = -1;
        if (b->withhold >= 0) {
            std::vector<double> cost(b->count);
            std::vector<int> ord(b->count);
            for (int d = 0; d < b->count; ++d) {
                cost[d] = solve_cost(tdg_plan_internal(b->plans[d]));
                ord[d] = d;
            }
            std::stable_sort(ord.begin(), ord.end(), [&](int x, int y) { return cost[x] > cost[y]; });
            for (int i = 0; i < b->count; ++i)
                if (ord[i] == b->withhold) dv.withhold = i;
        }
        e = launch_batched_net(dv, b->nblocks, s);
    } else if (e == cudaSuccess) {
        BatchDev dv;
        dv.disks = b->disks;
        dv.start = b->start;
        dv.done = b->done;
        dv.ticket = b->done + kPhases * b->count;
        dv.err = b->err;
        dv.count = b->count;
        dv.total = b->total;
        dv.withhold = b->withhold;
        k_batched<<<b->blocks, b->threads, b->smem, s>>>(dv);
        e = cudaGetLastError();
    }
    if (prev >= 0) cudaSetDevice(prev);
    return e == cudaSuccess ? TDG_OK : TDG_ERR_CUDA;
}

tdg_status tdg_batch_debug_withhold(tdg_batch b, int grid) {
    if (!b || grid < -1 || grid >= b->count) return TDG_ERR_INVALID_ARG;
    b->withhold = grid;
    return TDG_OK;
}

tdg_status tdg_batch_get_error(tdg_batch b) {
    if (!b) return TDG_ERR_INVALID_ARG;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    int v = 0;
    cudaError_t e = cudaMemcpy(&v, b->err, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess && v != 0) e = cudaMemset(b->err, 0, sizeof(int));
    if (prev >= 0) cudaSetDevice(prev);
    if (e != cudaSuccess) return TDG_ERR_CUDA;
    return (tdg_status)v;
}

tdg_status tdg_batch_info(const tdg_batch b, int* blocks, int* threads, int* items, int* radix_pref) {
    if (!b) return TDG_ERR_INVALID_ARG;
    if (blocks) *blocks = b->threads == 64 ? b->nblocks : b->blocks;
    if (threads) *threads = b->threads;
    if (items) *items = b->threads == 64 ? b->ntotal : b->total;
    if (radix_pref) *radix_pref = b->radix_pref;
    return TDG_OK;
}

tdg_status tdg_batch_destroy(tdg_batch b) {
    if (!b) return TDG_ERR_INVALID_ARG;
    int prev = -1;
    cudaGetDevice(&prev);
    cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    batch_free(b);
    if (prev >= 0) cudaSetDevice(prev);
    delete b;
    return TDG_OK;
}

}  // extern "C"
