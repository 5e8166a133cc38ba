// Host side of the Krylov-projected step (Sec. 2.1): co-resident capacity
// and thread-block clusters per device, the probe and check of cluster
// formation, the launches of the single-run and batched kernels, dispatched
// by bulk type and DD order (the kernels are compiled per DD order in
// krylov_p2.cu, krylov_p3.cu and krylov_p4.cu from krylov_impl.cuh).
#include <cooperative_groups.h>

#include <cstdlib>
#include <mutex>

#include "kernels.h"

namespace wrc {

namespace {
constexpr int kPT = 128;      // threads per block of the single-run kernel
constexpr int kOutP = 66;     // partial sums per block (as in krylov_impl.cuh)

// Cluster formation check: launched with the attributes of the clustered
// Krylov kernel (cooperative, clusters of CL blocks, grid of one cluster),
// block 0 records how many blocks its cluster holds.  Reads no peer memory.
__global__ void k_cluster_probe(int* out) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *out = (int)cooperative_groups::this_cluster().num_blocks();
}

// Calls f with the KrylovKernels<T, P> of DD half-order P (2, 3 or 4).
template <typename T, typename F>
auto by_order(int P, F&& f) {
    if (P == 3) return f(KrylovKernels<T, 3>{});
    if (P == 4) return f(KrylovKernels<T, 4>{});
    return f(KrylovKernels<T, 2>{});
}
}  // namespace

namespace {
// Per device: whether clusters of 2 and 4 blocks form on the launch path
// (probe), whether a clustered launch has been checked, and per bulk type and
// DD order the co-resident blocks of the single-run kernel for clusters of
// 1, 2 and 4 blocks (0 where that cluster size cannot be launched
// cooperatively or does not form).
constexpr int kMaxDevices = 64;
struct ClusterCaps {
    bool ready = false;
    int cap[3] = {0, 0, 0};
};
struct DeviceClusters {
    bool probed = false;
    bool formed[3] = {true, false, false};   // [log2 CL]
    bool checked = false;
    ClusterCaps caps[2][kMaxP + 1];          // [fp32][P]
};
DeviceClusters g_dev[kMaxDevices];
std::mutex g_caps_mutex;
// Test switch (environment variable WRC_KRYLOV_TEST_REFUSE=1, read once per
// process): the first, checked clustered launch on a device behaves as if
// its clusters were not formed, so that the fallback path can be tested on
// a launch path that does form them.
int g_test_refuse = -1;

// Launch the probe as one cluster of CL blocks with the Krylov kernel's
// attributes and report whether the cluster formed (1), did not (0), or the
// launch failed (-1).  Runs on a short-lived stream of its own.
int probe_cluster(int CL) {
    int* d = nullptr;
    cudaStream_t ps = nullptr;
    if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    int r = -1;
    if (cudaStreamCreateWithFlags(&ps, cudaStreamNonBlocking) == cudaSuccess &&
        cudaMemsetAsync(d, 0, sizeof(int), ps) == cudaSuccess) {
        cudaLaunchConfig_t cfg = {};
        cudaLaunchAttribute at[2];
        at[0].id = cudaLaunchAttributeCooperative;
        at[0].val.cooperative = 1;
        at[1].id = cudaLaunchAttributeClusterDimension;
        at[1].val.clusterDim.x = CL;
        at[1].val.clusterDim.y = 1;
        at[1].val.clusterDim.z = 1;
        cfg.gridDim = dim3(CL);
        cfg.blockDim = dim3(32);
        cfg.stream = ps;
        cfg.attrs = at;
        cfg.numAttrs = 2;
        int h = 0;
        if (cudaLaunchKernelEx(&cfg, k_cluster_probe, d) == cudaSuccess &&
            cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, ps) == cudaSuccess &&
            cudaStreamSynchronize(ps) == cudaSuccess) {
            note_launch();
            r = h == CL ? 1 : 0;
        }
    }
    if (r < 0) cudaGetLastError();
    if (ps) cudaStreamDestroy(ps);
    cudaFree(d);
    return r;
}

// Cluster size for a launch of `blocks` blocks: the largest of 4 and 2 (at
// most cmax) that divides it within the co-resident capacity, else 1.
int cluster_for(const ClusterCaps& c, int blocks, int cmax) {
    if (cmax >= 4 && blocks % 4 == 0 && blocks <= c.cap[2]) return 4;
    if (cmax >= 2 && blocks % 2 == 0 && blocks <= c.cap[1]) return 2;
    return 1;
}

int clamp_order(int P) { return P == 3 || P == 4 ? P : 2; }

ClusterCaps caps_of(int dev, bool fp32, int P) {
    std::lock_guard<std::mutex> lk(g_caps_mutex);
    return (dev >= 0 && dev < kMaxDevices) ? g_dev[dev].caps[fp32][clamp_order(P)] : ClusterCaps{};
}

bool cluster_checked(int dev) {
    std::lock_guard<std::mutex> lk(g_caps_mutex);
    return dev >= 0 && dev < kMaxDevices && g_dev[dev].checked;
}
}  // namespace

int krylov_cluster_max() {
    // WRC_KRYLOV_CLUSTER = 1 or 2 caps the cluster size (default 4)
    int cmax = 4;
    if (const char* ev = getenv("WRC_KRYLOV_CLUSTER")) cmax = atoi(ev) >= 4 ? 4 : (atoi(ev) >= 2 ? 2 : 1);
    return cmax;
}

int krylov_step_init(int dev, bool fp32, int P, int* max_blocks) {
    if (dev < 0 || dev >= kMaxDevices) return -1;
    P = clamp_order(P);
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const cudaError_t e = fp32 ? by_order<float>(P, [&](auto K) { return K.occupancy(&per); })
                               : by_order<double>(P, [&](auto K) { return K.occupancy(&per); });
    if (e != cudaSuccess || per < 1) return -2;
    *max_blocks = sms * per;
    std::lock_guard<std::mutex> lk(g_caps_mutex);
    if (g_test_refuse < 0) {
        const char* ev = getenv("WRC_KRYLOV_TEST_REFUSE");
        g_test_refuse = (ev && atoi(ev) == 1) ? 1 : 0;
    }
    DeviceClusters& D = g_dev[dev];
    if (!D.probed) {
        // a launch path that does not form clusters (some profilers replay a
        // cooperative launch without them): use the unclustered kernel
        D.formed[1] = probe_cluster(2) == 1;
        D.formed[2] = probe_cluster(4) == 1;
        D.probed = true;
    }
    ClusterCaps& c = D.caps[fp32][P];
    if (c.ready) return 0;
    c.cap[0] = sms * per;
    for (int q = 1; q <= 2; ++q)
        c.cap[q] = !D.formed[q] ? 0
                   : fp32 ? by_order<float>(P, [&](auto K) { return K.cluster_capacity(1 << q); })
                          : by_order<double>(P, [&](auto K) { return K.cluster_capacity(1 << q); });
    c.ready = true;
    return 0;
}

int krylov_step_blocks(long long n, int max_blocks, bool fp32, int P, int dev, int cmax) {
    const ClusterCaps c = caps_of(dev, fp32, P);
    long long b = (n + kPT - 1) / kPT;
    if (b < 1) b = 1;
    if (b > max_blocks) b = max_blocks;
    // padded to a whole number of clusters where that fits (the extra blocks
    // have no points and contribute zero partial sums)
    const long long b4 = (b + 3) / 4 * 4, b2 = (b + 1) / 2 * 2;
    if (cmax >= 4 && b4 <= c.cap[2] && b4 <= max_blocks) return (int)b4;
    if (cmax >= 2 && b2 <= c.cap[1] && b2 <= max_blocks) return (int)b2;
    return (int)b;
}

int krylov_step_cluster(long long n, int max_blocks, bool fp32, int P, int dev, int cmax) {
    return cluster_for(caps_of(dev, fp32, P), krylov_step_blocks(n, max_blocks, fp32, P, dev, cmax), cmax);
}

void krylov_clusters_unformed(int dev) {
    if (dev < 0 || dev >= kMaxDevices) return;
    std::lock_guard<std::mutex> lk(g_caps_mutex);
    DeviceClusters& D = g_dev[dev];
    D.checked = true;
    D.formed[1] = D.formed[2] = false;
    for (auto& byp : D.caps)
        for (auto& cc : byp) cc.cap[1] = cc.cap[2] = 0;
}

// The first clustered launch on a device is checked: the stream is
// synchronised and, if the kernel found its clusters not formed (it then
// runs as the unclustered kernel and raises bit 4 of the error word),
// clusters are switched off for the device.  Later launches are not
// synchronised; a later launch without its clusters (e.g. under a profiler)
// runs unclustered all the same and is seen at the step's host
// synchronisation.
template <typename T>
cudaError_t launch_krylov_step(const KrylovStepArgs& args, int blocks, cudaStream_t s, int dev, int cmax) {
    const bool fp32 = sizeof(T) == 4;
    const int P = clamp_order(args.g.P);
    const ClusterCaps c = caps_of(dev, fp32, P);
    const int cl = cluster_for(c, blocks, cmax);
    const bool check = cl > 1 && !cluster_checked(dev);
    KrylovStepArgs a = args;
    a.refuse = (check && g_test_refuse == 1) ? 1 : 0;
    cudaError_t e = by_order<T>(P, [&](auto K) { return K.launch(a, blocks, cl, s); });
    if (e != cudaSuccess) return e;
    note_launch();
    e = cudaGetLastError();
    if (e != cudaSuccess || !check) return e;
    int err = 0;
    e = cudaMemcpyAsync(&err, args.err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return e;
    if (err & 16) {
        krylov_clusters_unformed(dev);
        if (err == 16) e = cudaMemsetAsync(args.err, 0, sizeof(int), s);   // informational only
    } else {
        std::lock_guard<std::mutex> lk(g_caps_mutex);
        g_dev[dev].checked = true;
    }
    return e;
}

template cudaError_t launch_krylov_step<double>(const KrylovStepArgs&, int, cudaStream_t, int, int);
template cudaError_t launch_krylov_step<float>(const KrylovStepArgs&, int, cudaStream_t, int, int);

size_t krylov_partials_doubles(int max_blocks) { return (size_t)3 * max_blocks * kOutP; }

int krylov_batch_max_blocks(bool fp32, int P, int pt, bool pair) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const void* k = fp32 ? by_order<float>(P, [&](auto K) { return K.batch_kernel(pt, pair); })
                         : by_order<double>(P, [&](auto K) { return K.batch_kernel(pt, pair); });
    if (!k) return -1;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k, pt, 0) != cudaSuccess || per < 1) return -2;
    return sms * per;
}

template <typename T>
cudaError_t launch_krylov_batch(const KrylovStepArgs* d_args, const int* d_blk2mem, const int* d_mem_b0,
                                int members, int blocks, int pt, int P, cudaStream_t s, bool pair) {
    void* params[] = {(void*)&d_args, (void*)&d_blk2mem, (void*)&d_mem_b0};
    const void* k = by_order<T>(P, [&](auto K) { return K.batch_kernel(pt, pair); });
    if (!k) return cudaErrorInvalidValue;
    cudaError_t e = cudaLaunchCooperativeKernel(k, dim3(blocks), dim3(pt), params, 0, s);
    if (e != cudaSuccess) return e;
    note_launch();
    (void)members;
    return cudaGetLastError();
}

template cudaError_t launch_krylov_batch<double>(const KrylovStepArgs*, const int*, const int*, int, int, int, int,
                                                 cudaStream_t, bool);
template cudaError_t launch_krylov_batch<float>(const KrylovStepArgs*, const int*, const int*, int, int, int, int,
                                                cudaStream_t, bool);

}  // namespace wrc
