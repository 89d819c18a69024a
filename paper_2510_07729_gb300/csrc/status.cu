// Device status word: kernels that meet a problem they cannot report through
// a return value (a non-finite input, an index out of range, a bake ray that
// stopped early) set a bit in one 32-bit word per device with atomicOr.
// sop_device_status() synchronises a stream and reads (and optionally clears)
// the word. The word is sticky: bits stay set until a caller clears them.
#include <atomic>
#include <stdio.h>
#include <string.h>

#include "sop_device.cuh"
#include "sop_internal.h"

namespace {

__device__ unsigned int g_status_word;

constexpr int kMaxDevices = 64;
std::atomic<unsigned int*> g_addr[kMaxDevices];

thread_local char g_msg[256];

}  // namespace

namespace sop {

unsigned int* status_word()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return nullptr;
    unsigned int* p = g_addr[dev].load(std::memory_order_acquire);
    if (p) return p;
    void* a = nullptr;
    if (cudaGetSymbolAddress(&a, g_status_word) != cudaSuccess || !a) return nullptr;
    g_addr[dev].store(static_cast<unsigned int*>(a), std::memory_order_release);
    return static_cast<unsigned int*>(a);
}

const char* status_bits_message(uint32_t bits)
{
    g_msg[0] = 0;
    size_t o = 0;
    auto add = [&](const char* s) {
        const size_t n = strlen(s);
        if (o + n + 3 >= sizeof(g_msg)) return;
        if (o) {
            memcpy(g_msg + o, "; ", 2);
            o += 2;
        }
        memcpy(g_msg + o, s, n + 1);
        o += n;
    };
    if (bits & SOP_DEVSTAT_NONFINITE) add("a non-finite input value (NaN or Inf) was met");
    if (bits & SOP_DEVSTAT_BAKE_TRUNCATED)
        add("a bake ray met more hits at one depth than its hit buffer holds and stopped there");
    if (bits & SOP_DEVSTAT_INDEX) add("an index outside its range was skipped");
    if (bits & SOP_DEVSTAT_CAPACITY) add("a fixed-capacity buffer overflowed (part of the input was used)");
    if (bits & SOP_DEVSTAT_TIMEOUT) add("a bounded wait for the tensor cores gave up (that launch's outputs are not valid)");
    if (bits & SOP_DEVSTAT_GRID_COARSENED) add("(info) the binning grid was coarsened to fit the workspace");
    return g_msg;
}

}  // namespace sop

namespace {

__device__ unsigned int g_status_taken;

__global__ void status_take_kernel(unsigned int* word, unsigned int* taken, int clear)
{
    *taken = clear ? atomicExch(word, 0u) : atomicOr(word, 0u);
}

}  // namespace

namespace sop {

cudaError_t status_take(uint32_t* host_out, bool clear, cudaStream_t s)
{
    unsigned int* w = status_word();
    if (!w) return cudaErrorInvalidDevice;
    void* t = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&t, g_status_taken);
    if (e != cudaSuccess) return e;
    status_take_kernel<<<1, 1, 0, s>>>(w, static_cast<unsigned int*>(t), clear ? 1 : 0);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(host_out, t, sizeof(uint32_t), cudaMemcpyDeviceToHost, s)) != cudaSuccess) return e;
    return cudaStreamSynchronize(s);
}

}  // namespace sop
