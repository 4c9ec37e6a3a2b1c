// Thin QR entry point that allocates nothing.
//
// Some callers cannot allocate device memory at the point where they need a
// QR: applications whose device memory is owned by a pool or arena (a
// framework's caching allocator that has reserved the free memory, an
// embedded deployment that forbids allocation after start-up), and
// latency-critical paths that must not risk the device-wide synchronisation
// that cudaMalloc and cudaFree can cause.  tucker_orth_noalloc serves them:
// its scratch is a fixed file-scope device array, so it needs no handle and
// no workspace, and it calls no cudaMalloc, cudaFree or allocating library
// routine.
#include <mutex>

#include "tk_internal.cuh"

namespace tk {
namespace {

// Largest sketch it accepts: rows <= kRowsMax, columns <= kColsMax.
constexpr int64_t kRowsMax = 4096;
constexpr int64_t kColsMax = 64;
// CholeskyQR2 + Householder scratch at that size, as the planning pass counts
// it: three rows x cols FP64 matrices (Q, the first CholeskyQR factor, the
// Householder copy: 6 MiB), the split-K partial tiles of the two Gram
// products (19 slices of 64 x 64 FP64 each at 4096 rows: 1.2 MB), two
// cols x cols FP64 matrices, the flag header and 256-byte alignment of every
// block: 7.3 MB, rounded up to 8 MiB.
constexpr size_t kScratchBytes = 8u << 20;

// Shared by every call on a device and kept between calls.
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

struct DeviceScratch {
    char* ptr = nullptr;
};
constexpr int kMaxDevices = 64;
DeviceScratch g_devices[kMaxDevices];
std::mutex g_mutex;

// Device address of g_scratch on the current device.  The host-side symbol is
// only a stand-in, so the address is looked up once per device with that
// device current.
tk_status scratch_for_current_device(char** out) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return TK_ERR_CUDA;
    std::lock_guard<std::mutex> lock(g_mutex);
    if (!g_devices[dev].ptr) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess) {
            cudaGetLastError();
            return TK_ERR_CUDA;
        }
        g_devices[dev].ptr = static_cast<char*>(p);
    }
    *out = g_devices[dev].ptr;
    return TK_OK;
}

}  // namespace
}  // namespace tk

using namespace tk;

extern "C" tk_status tucker_orth_noalloc(void* cuda_stream, const tk_matrix* Y, tk_matrix* Q, int* info) {
    try {
        Mat y = mat_in(Y, "Y");
        Mat q = mat_in(Q, "Q");
        if (!(y.dt == TK_F64 || y.dt == TK_F32) || !(q.dt == TK_F64 || q.dt == TK_F32)) return TK_ERR_DTYPE;
        const int64_t k = std::min(y.rows, y.cols);
        if (q.rows != y.rows || q.cols != k) return TK_ERR_SHAPE;
        if (y.rows > kRowsMax || k > kColsMax) return TK_ERR_SHAPE;  // beyond the fixed scratch
        // the scratch address and the launches belong to the current device: the stream must be one of its own
        int cur = 0, sdev = 0;
        TK_CUDA(cudaGetDevice(&cur));
        TK_CUDA(cudaStreamGetDevice(static_cast<cudaStream_t>(cuda_stream), &sdev));
        if (sdev != cur) return TK_ERR_ARG;
        // reading info back synchronises the stream, which a stream recording a CUDA graph must not do
        cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
        TK_CUDA(cudaStreamIsCapturing(static_cast<cudaStream_t>(cuda_stream), &cap));
        if (info && cap != cudaStreamCaptureStatusNone) return TK_ERR_ARG;
        char* base = nullptr;
        tk_status st = scratch_for_current_device(&base);
        if (st != TK_OK) return st;
        // flags at the start of the scratch; the rest is handed out by the bump allocator
        Ctx plan;
        plan.exec = false;
        plan.used = 256;
        orth_matrix(plan, y, q);
        if (plan.used > kScratchBytes) return TK_ERR_SHAPE;
        Ctx c;
        c.exec = true;
        c.stream = static_cast<cudaStream_t>(cuda_stream);
        c.base = base;
        c.used = 256;
        c.dflags = reinterpret_cast<unsigned*>(base);
        c.dqr = reinterpret_cast<int*>(base + 16);
        orth_matrix(c, y, q);
        if (info) {
            TK_CUDA(cudaMemcpyAsync(info, c.dqr, sizeof(int), cudaMemcpyDeviceToHost, c.stream));
            TK_CUDA(cudaStreamSynchronize(c.stream));
        }
        return TK_OK;
    } catch (const Error& e) {
        return e.st;
    } catch (...) {
        return TK_ERR_ARG;
    }
}
