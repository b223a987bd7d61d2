// Test support only: runs the library's bounded waits -- the mbarrier wait
// (mbar_wait_bounded, used by the tensor-core pass for its products) on a
// barrier that nothing arrives at and on one whose phase has completed, and
// the counter wait (flag_wait_bounded, used by the persistent ensemble
// kernel for its dependencies) on a counter below, at its target and with
// the abort word set -- so a test can check that each wait gives up after its
// limit, reports it, and leaves the context usable.
#include "../paper_1608_00263_gb300/csrc/qs_device.cuh"

__global__ void k_wait_probe(unsigned long long limit_ns, int arrive, int *ok, unsigned long long *elapsed)
{
    __shared__ __align__(8) unsigned long long bar;
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(&bar);
    if (threadIdx.x == 0) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(a) : "memory");
    __syncthreads();
    if (arrive && threadIdx.x == 0)
        asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.shared::cta.b64 st, [%0];\n}" ::"r"(a) : "memory");
    __syncthreads();
    unsigned long long t0, t1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    const bool done = qs::mbar_wait_bounded(a, 0, limit_ns);
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
    if (threadIdx.x == 0) {
        *ok = done ? 1 : 0;
        *elapsed = t1 - t0;
    }
}

extern "C" int wait_probe(unsigned long long limit_ns, int arrive, int *ok, unsigned long long *elapsed_ns)
{
    int *d_ok = nullptr;
    unsigned long long *d_el = nullptr;
    cudaError_t e = cudaMalloc((void **)&d_ok, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&d_el, sizeof(unsigned long long));
    if (e == cudaSuccess) {
        k_wait_probe<<<1, 32>>>(limit_ns, arrive, d_ok, d_el);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(ok, d_ok, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(elapsed_ns, d_el, sizeof(unsigned long long), cudaMemcpyDeviceToHost);
    cudaFree(d_ok);
    cudaFree(d_el);
    return (int)e;
}

// The persistent ensemble kernel's dependency wait (flag_wait_bounded) on a
// global counter: `value` is the counter (target 1), `abort` the abort word.
__global__ void k_flag_probe(unsigned long long limit_ns, unsigned int *words, int *ret,
                             unsigned long long *elapsed)
{
    unsigned long long t0, t1;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    const int r = qs::flag_wait_bounded(words, 1u, words + 1, limit_ns);
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t1));
    if (threadIdx.x == 0) {
        *ret = r;
        *elapsed = t1 - t0;
    }
}

extern "C" int flag_probe(unsigned long long limit_ns, unsigned int value, unsigned int abort, int *ret,
                          unsigned long long *elapsed_ns)
{
    unsigned int *d_w = nullptr;
    int *d_r = nullptr;
    unsigned long long *d_el = nullptr;
    const unsigned int h_w[2] = {value, abort};
    cudaError_t e = cudaMalloc((void **)&d_w, sizeof h_w);
    if (e == cudaSuccess) e = cudaMalloc((void **)&d_r, sizeof(int));
    if (e == cudaSuccess) e = cudaMalloc((void **)&d_el, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMemcpy(d_w, h_w, sizeof h_w, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) {
        k_flag_probe<<<1, 32>>>(limit_ns, d_w, d_r, d_el);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(ret, d_r, sizeof(int), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(elapsed_ns, d_el, sizeof(unsigned long long), cudaMemcpyDeviceToHost);
    cudaFree(d_w);
    cudaFree(d_r);
    cudaFree(d_el);
    return (int)e;
}
