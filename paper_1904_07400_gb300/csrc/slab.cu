// The slab decomposition of one grid over `world` ranks (Sec. 2.3 splits the spline solves
// and the transforms over processes in slabs, with transposes between the passes).
//
// Rank r owns rows [r0, r0 + nrows) of sigma and of the forces, and the two-column tiles
// [t0, t0 + ntiles) of frequency columns (ky = 2 t0 .. 2 (t0 + ntiles) - 1, the last rank
// ending at the Nyquist column ky = L).  One solve is
//   1. pass A on the rank's rows:               sigma rows -> Z row slab [tile][row pos]
//   2. all-to-all: the chunk for rank q is tiles [t0_q, t0_q + ntiles_q) of the Z row slab,
//      contiguous; rank q receives one chunk per source, in source order
//   3. tdg_slab_unpack_z: received chunks -> Z column slab [tile - t0][position of row]
//   4. pass B on the rank's columns:            Z column slab -> G column slab
//   5. tdg_slab_pack_g: G column slab -> one chunk per destination r (its rows of every
//      local tile), per component
//   6. all-to-all per component: rank r receives, in source order, exactly its G row slab
//   7. pass C on the rank's rows:               G row slab -> force rows
// Cells (16 bytes: two complex floats of adjacent columns) are the unit of every layout and
// of every split size.  Steps 3 and 5 are 2-D device copies (cudaMemcpy2DAsync), on the
// receiving or sending rank's own memory; the transport of steps 2 and 6 is the caller's
// (NCCL or gloo all-to-all, or plain copies when several ranks share one device).
#include <cuda_runtime.h>

#include <algorithm>

#include "tdg_internal.cuh"

namespace {

using tdg::Plan;

int ntile_of(const Plan& p) { return (p.hy + 1) / 2; }

// rows in multiples of 16 (the order >= 3 row permutation works on 16-row chunks), the
// extra chunks to the first ranks; tiles evenly, the extra ones to the first ranks
void partition(int nx, int ntile, int world, int rank, int* r0, int* nrows, int* t0, int* ntiles) {
    const int chunks = nx / 16, cq = chunks / world, cr = chunks % world;
    *r0 = 16 * (rank * cq + std::min(rank, cr));
    *nrows = 16 * (cq + (rank < cr ? 1 : 0));
    const int tq = ntile / world, tr = ntile % world;
    *t0 = rank * tq + std::min(rank, tr);
    *ntiles = tq + (rank < tr ? 1 : 0);
}

bool slab_ok(const Plan& p, int world, int rank) {
    return p.built && p.prec == TDG_FP32 && p.spec_half && p.net_tw && world >= 1 && rank >= 0 && rank < world &&
           p.nx % 16 == 0 && p.nx / 16 >= world && ntile_of(p) >= world;
}

struct Guard {
    int prev = -1;
    bool ok = false;
    explicit Guard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~Guard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

bool al16(const void* a) { return ((uintptr_t)a & 15u) == 0; }

tdg_status status_of(cudaError_t e) { return e == cudaSuccess ? TDG_OK : TDG_ERR_CUDA; }

}  // namespace

extern "C" {

tdg_status tdg_slab_partition(int nx, int ny, int world, int rank, int* r0, int* nrows, int* t0, int* ntiles) {
    const int ly = tdg::net_fp32_length(ny);
    if (!tdg::net_fp32_length(nx) || !ly || world < 1 || rank < 0 || rank >= world || nx / 16 < world)
        return TDG_ERR_INVALID_ARG;
    const int ntile = (ly + 2) / 2;  // hy = ly + 1 columns
    if (ntile < world) return TDG_ERR_INVALID_ARG;
    int a, b, c, d;
    partition(nx, ntile, world, rank, &a, &b, &c, &d);
    if (r0) *r0 = a;
    if (nrows) *nrows = b;
    if (t0) *t0 = c;
    if (ntiles) *ntiles = d;
    return TDG_OK;
}

size_t tdg_slab_bytes(const tdg_plan h, int world, int rank, int which) {
    if (!h) return 0;
    const Plan& p = tdg_plan_internal(h);
    if (!slab_ok(p, world, rank) || which < 0 || which > 3) return 0;
    int r0, nrows, t0, ntiles;
    partition(p.nx, ntile_of(p), world, rank, &r0, &nrows, &t0, &ntiles);
    const size_t cell = tdg::kSlabCell;
    switch (which) {
        case 0: return (size_t)ntile_of(p) * nrows * cell;      // Z row slab (= send chunks)
        case 1: return (size_t)ntiles * p.nx * cell;            // Z column slab (= received chunks)
        case 2: return 2 * (size_t)ntiles * p.nx * cell;        // G column slab (= G send chunks)
        default: return 2 * (size_t)ntile_of(p) * nrows * cell; // G row slab (= received chunks)
    }
}

tdg_status tdg_slab_rows_forward(tdg_plan h, int world, int rank, const void* sigma_rows, void* z_rows,
                                 tdg_stream stream) {
    if (!h || !sigma_rows || !z_rows || !al16(sigma_rows) || !al16(z_rows)) return TDG_ERR_INVALID_ARG;
    const Plan& p = tdg_plan_internal(h);
    if (!p.built) return TDG_ERR_NOT_BUILT;
    if (!slab_ok(p, world, rank)) return TDG_ERR_UNSUPPORTED;
    int r0, nrows, t0, ntiles;
    partition(p.nx, ntile_of(p), world, rank, &r0, &nrows, &t0, &ntiles);
    Guard g(p.device);
    if (!g.ok) return TDG_ERR_CUDA;
    return status_of(tdg::launch_slab_rows(p, static_cast<const float*>(sigma_rows), nrows, z_rows,
                                           reinterpret_cast<cudaStream_t>(stream)));
}

tdg_status tdg_slab_unpack_z(tdg_plan h, int world, int rank, const void* recv, void* z_cols, tdg_stream stream) {
    if (!h || !recv || !z_cols || !al16(recv) || !al16(z_cols)) return TDG_ERR_INVALID_ARG;
    const Plan& p = tdg_plan_internal(h);
    if (!p.built) return TDG_ERR_NOT_BUILT;
    if (!slab_ok(p, world, rank)) return TDG_ERR_UNSUPPORTED;
    int r0, nrows, t0, ntiles;
    partition(p.nx, ntile_of(p), world, rank, &r0, &nrows, &t0, &ntiles);
    Guard g(p.device);
    if (!g.ok) return TDG_ERR_CUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t cell = tdg::kSlabCell;
    const bool rowmap = tdg::solve_order(p) != 0;  // rows at (i % 16) (nx / 16) + i / 16
    const char* src = static_cast<const char*>(recv);
    char* dst = static_cast<char*>(z_cols);
    for (int q = 0; q < world; ++q) {
        int qr0, qn, qt0, qnt;
        partition(p.nx, ntile_of(p), world, q, &qr0, &qn, &qt0, &qnt);
        // chunk of source q: [tile - t0][q's row position], q's rows permuted within its slab
        if (rowmap) {
            for (int res = 0; res < 16; ++res) {
                cudaError_t e = cudaMemcpy2DAsync(dst + ((size_t)res * (p.nx / 16) + qr0 / 16) * cell, p.nx * cell,
                                                  src + (size_t)res * (qn / 16) * cell, qn * cell, (qn / 16) * cell,
                                                  ntiles, cudaMemcpyDeviceToDevice, s);
                if (e != cudaSuccess) return TDG_ERR_CUDA;
            }
        } else {
            cudaError_t e = cudaMemcpy2DAsync(dst + (size_t)qr0 * cell, p.nx * cell, src, qn * cell, qn * cell,
                                              ntiles, cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return TDG_ERR_CUDA;
        }
        src += (size_t)ntiles * qn * cell;
    }
    return TDG_OK;
}

tdg_status tdg_slab_columns(tdg_plan h, int world, int rank, const void* z_cols, void* g_cols, tdg_stream stream) {
    if (!h || !z_cols || !g_cols || !al16(z_cols) || !al16(g_cols)) return TDG_ERR_INVALID_ARG;
    const Plan& p = tdg_plan_internal(h);
    if (!p.built) return TDG_ERR_NOT_BUILT;
    if (!slab_ok(p, world, rank)) return TDG_ERR_UNSUPPORTED;
    int r0, nrows, t0, ntiles;
    partition(p.nx, ntile_of(p), world, rank, &r0, &nrows, &t0, &ntiles);
    const int ky0 = 2 * t0, nky = std::min(2 * (t0 + ntiles), p.hy) - ky0;
    Guard g(p.device);
    if (!g.ok) return TDG_ERR_CUDA;
    return status_of(tdg::launch_slab_cols(p, z_cols, ky0, nky, ntiles, g_cols, reinterpret_cast<cudaStream_t>(stream)));
}

tdg_status tdg_slab_pack_g(tdg_plan h, int world, int rank, const void* g_cols, void* send, tdg_stream stream) {
    if (!h || !g_cols || !send || !al16(g_cols) || !al16(send)) return TDG_ERR_INVALID_ARG;
    const Plan& p = tdg_plan_internal(h);
    if (!p.built) return TDG_ERR_NOT_BUILT;
    if (!slab_ok(p, world, rank)) return TDG_ERR_UNSUPPORTED;
    int r0, nrows, t0, ntiles;
    partition(p.nx, ntile_of(p), world, rank, &r0, &nrows, &t0, &ntiles);
    Guard g(p.device);
    if (!g.ok) return TDG_ERR_CUDA;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const size_t cell = tdg::kSlabCell;
    const size_t comp = (size_t)ntiles * p.nx * cell;  // one component, in both buffers
    for (int c = 0; c < 2; ++c) {
        const char* src = static_cast<const char*>(g_cols) + c * comp;
        char* dst = static_cast<char*>(send) + c * comp;
        for (int q = 0; q < world; ++q) {
            int qr0, qn, qt0, qnt;
            partition(p.nx, ntile_of(p), world, q, &qr0, &qn, &qt0, &qnt);
            // chunk for rank q: [tile - t0][q's rows, natural order]
            cudaError_t e = cudaMemcpy2DAsync(dst, qn * cell, src + (size_t)qr0 * cell, p.nx * cell, qn * cell,
                                              ntiles, cudaMemcpyDeviceToDevice, s);
            if (e != cudaSuccess) return TDG_ERR_CUDA;
            dst += (size_t)ntiles * qn * cell;
        }
    }
    return TDG_OK;
}

tdg_status tdg_slab_rows_inverse(tdg_plan h, int world, int rank, const void* g_rows, void* fx_rows, void* fy_rows,
                                 tdg_stream stream) {
    if (!h || !g_rows || !fx_rows || !fy_rows || !al16(g_rows) || !al16(fx_rows) || !al16(fy_rows) ||
        fx_rows == fy_rows)
        return TDG_ERR_INVALID_ARG;
    const Plan& p = tdg_plan_internal(h);
    if (!p.built) return TDG_ERR_NOT_BUILT;
    if (!slab_ok(p, world, rank)) return TDG_ERR_UNSUPPORTED;
    int r0, nrows, t0, ntiles;
    partition(p.nx, ntile_of(p), world, rank, &r0, &nrows, &t0, &ntiles);
    Guard g(p.device);
    if (!g.ok) return TDG_ERR_CUDA;
    return status_of(tdg::launch_slab_rows_inv(p, g_rows, nrows, static_cast<float*>(fx_rows),
                                               static_cast<float*>(fy_rows), reinterpret_cast<cudaStream_t>(stream)));
}

}  // extern "C"
