// tdg_solve_forces_noalloc: the force solve with its scratch in a fixed, file-scope
// device array instead of a cudaMalloc'd workspace.
//
// Who needs it: tdg_solve_forces allocates the plan's workspace on its first call (unless
// the caller handed one over with tdg_set_workspace).  Some callers cannot allocate at
// the point where they solve: code running while another allocator owns the device's
// free memory, real-time loops that must not hit cudaMalloc's implicit device
// synchronisation, or hosts that forbid device allocations after start-up.  They build
// their plans up front and solve through this entry point, which allocates nothing.
//
// The scratch lives in the static array below (kNoallocScratchBytes = 32 MiB).  Every GPU
// that loads the library holds that array until the process exits.  Every call shares
// it and it keeps the last call's contents; nothing in it has to start at zero, because
// each pass writes every element the next pass reads.  Calls that overlap on the GPU
// (other streams, other host threads) race on the array and must be serialised by the
// caller.
#include <cuda_runtime.h>

#include "tdg_internal.cuh"

namespace {

constexpr size_t kNoallocScratchBytes = TDG_NOALLOC_SCRATCH_BYTES;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

}  // namespace

namespace tdg {
// Device address of the scratch array on the current device.  In host code the array's
// name is only a host-side stand-in, so the address must come from cudaGetSymbolAddress.
// Called when a plan's kernel tables are built (outside any stream capture), with the plan's
// device current; the plan keeps the address, so a solve makes no set-up call and a plan
// never outlives the context it was looked up in.
cudaError_t noalloc_scratch(void** out) { return cudaGetSymbolAddress(out, g_noalloc_scratch); }
}  // namespace tdg

extern "C" tdg_status tdg_solve_forces_noalloc(tdg_plan h, const void* sigma, void* fx, void* fy,
                                               tdg_stream stream) {
    using namespace tdg;
    if (!h) return TDG_ERR_INVALID_ARG;
    const Plan& p = tdg_plan_internal(h);
    if (!sigma || !fx || !fy || (((uintptr_t)sigma | (uintptr_t)fx | (uintptr_t)fy) & 15u))
        return TDG_ERR_INVALID_ARG;
    if (fx == fy || fx == sigma || fy == sigma) return TDG_ERR_INVALID_ARG;
    if (!p.built) return TDG_ERR_NOT_BUILT;
    if (workspace_bytes(p) > kNoallocScratchBytes) return TDG_ERR_UNSUPPORTED;
    if (!p.noalloc) return TDG_ERR_CUDA;  // the address lookup at build time failed
    int prev = -1;
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    if (cudaSetDevice(p.device) != cudaSuccess) return TDG_ERR_CUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    cudaError_t e;
    if (p.prec == TDG_FP64)
        e = launch_forward<double>(p, (const double*)sigma, (double*)fx, (double*)fy, p.noalloc, s);
    else
        e = launch_forward<float>(p, (const float*)sigma, (float*)fx, (float*)fy, p.noalloc, s);
    if (prev >= 0) cudaSetDevice(prev);
    return e == cudaSuccess ? TDG_OK : TDG_ERR_CUDA;
}
