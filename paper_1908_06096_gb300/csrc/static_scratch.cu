// st_inv_trans_static: the inverse transform with its scratch in a fixed,
// file-scope device array instead of the plan's workspace.
//
// Who needs it: code that cannot allocate device memory at the point where it
// runs the transform -- hard real-time loops where an allocation could stall,
// or host frameworks that own all device memory through their own allocator
// and do not let components call cudaMalloc or cudaFree.  This entry point
// calls neither, nor any other allocating routine; the scratch it needs (the
// packed spectral operand and the Fourier buffer) comes from g_static_scratch
// below.
#include "st_internal.cuh"

#include <mutex>

namespace {

// Scratch shared by every call of st_inv_trans_static on a device.  It is
// part of the module image, so every GPU that loads the library holds these
// ST_STATIC_SCRATCH_BYTES until the process exits.
constexpr size_t ST_STATIC_SCRATCH_BYTES = 32u << 20;  // 32 MiB
static __device__ __align__(256) unsigned char g_static_scratch[ST_STATIC_SCRATCH_BYTES];

// Device address of g_static_scratch, looked up once per device and kept for
// the life of the process (the name g_static_scratch is only a host-side
// stand-in in host code; giving it to a kernel would hand the kernel the
// wrong memory).
constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
void *g_scratch_ptr[kMaxDevices] = {nullptr};

st_status scratch_address(void **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return st::cuda_fail(e, "cudaGetDevice");
    if (dev < 0 || dev >= kMaxDevices) {
        st::set_last_error("device index beyond the static-scratch table");
        return ST_ERR_UNSUPPORTED;
    }
    std::lock_guard<std::mutex> lock(g_scratch_mutex);
    if (!g_scratch_ptr[dev]) {
        void *ptr = nullptr;
        e = cudaGetSymbolAddress(&ptr, g_static_scratch);
        if (e != cudaSuccess) return st::cuda_fail(e, "cudaGetSymbolAddress(g_static_scratch)");
        g_scratch_ptr[dev] = ptr;
    }
    *out = g_scratch_ptr[dev];
    return ST_OK;
}

size_t align256(size_t n) { return (n + 255) & ~(size_t)255; }

}  // namespace

using namespace st;

extern "C" st_status st_inv_trans_static(st_plan_t p, const void *spec_dev, void *grid_dev, int nfields, void *stream)
{
    if (!p || !spec_dev || !grid_dev) return ST_ERR_ARG;
    if (nfields < 1) {
        set_last_error("nfields must be at least 1");
        return ST_ERR_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    const int Cp = cols_padded(nfields);
    const int store = store_of(p->prec);
    const size_t sop_bytes = align256((size_t)p->srow_total * Cp * store_bytes(store) * store_planes(store));
    const size_t fb_bytes = align256((size_t)fb_rows(p) * Cp * (p->prec == P_FP64 ? 8 : 4));
    if (sop_bytes + fb_bytes > ST_STATIC_SCRATCH_BYTES) {
        set_last_error("st_inv_trans_static: this plan and field count need " + std::to_string(sop_bytes + fb_bytes) +
                       " bytes of scratch; the static scratch holds " + std::to_string(ST_STATIC_SCRATCH_BYTES));
        return ST_ERR_ARG;
    }
    void *base = nullptr;
    st_status r = scratch_address(&base);
    if (r != ST_OK) return r;
    unsigned char *sop = (unsigned char *)base;
    unsigned char *fb = sop + sop_bytes;
    // The operand rows a GEMM tile reads past its own group meet zero table
    // entries, so they must hold finite values; the array keeps whatever the
    // previous call (possibly another plan or precision) left there, so the
    // operand region is cleared first.  The Fourier-buffer region needs no
    // clearing: the FFT reads only entries this call writes.
    ST_CUDA(cudaMemsetAsync(sop, 0, sop_bytes, s));
    // counted and timed with the plan's other launches
    if ((r = count_launch(p, K_PACK, s, [&] { return launch_pack(p, spec_dev, nfields, s, sop); }))) return r;
    r = count_launch(p, K_LEG_INV, s, [&] {
        return prec_is_tc(p->prec) ? launch_leg_tc(p, 0, nfields, s, sop, fb) : launch_leg_simt(p, 0, nfields, s, sop, fb);
    });
    if (r) return r;
    return count_launch(p, K_FFT_INV, s, [&] { return launch_fft_inv(p, grid_dev, nfields, s, fb); });
}

extern "C" size_t st_static_scratch_bytes(void) { return ST_STATIC_SCRATCH_BYTES; }
