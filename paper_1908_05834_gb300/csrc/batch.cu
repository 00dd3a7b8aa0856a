// bchar_step_batch: one time step of several independent meshes at once.
//
// Small meshes leave most of the GPU idle: a 64x64 step is a few hundred
// short kernels separated by host round trips (reading the number of
// non-zeros, building the multigrid levels, polling the conjugate gradients).
// Stepping many such handles one after the other keeps the GPU mostly idle;
// stepping them from concurrent host threads, each handle on its own stream,
// overlaps their kernels and their round trips.
//
// Each instance runs exactly the kernels, in exactly the order, of a plain
// bchar_step on its own stream, so a batched result is bitwise identical to
// the plain one.  The instances are handed to the workers largest first
// (cells), which packs uneven sizes onto the workers.
#include <algorithm>
#include <atomic>
#include <exception>
#include <numeric>
#include <thread>
#include <vector>

#include "internal.cuh"

using namespace bchar;

namespace {

constexpr int kDefaultWorkers = 16;

}  // namespace

extern "C" bchar_status bchar_step_batch(int count, const bchar_mesh_t *meshes, const double *dt,
                                         const void *const *c_in, void *const *c_out, const int *c_dtype,
                                         bchar_step_info *infos, bchar_status *statuses, int max_workers) {
    if (count < 0) return BCHAR_ERR_INVALID_ARG;
    if (count == 0) return BCHAR_OK;
    if (!meshes || !dt || !c_in || !c_out || !c_dtype) return BCHAR_ERR_INVALID_ARG;
    int caller_device = 0;
    if (cudaGetDevice(&caller_device) != cudaSuccess) {
        cudaGetLastError();
        return BCHAR_ERR_CUDA;
    }
    try {
        std::vector<bchar_mesh_t> handles(meshes, meshes + count);
        for (bchar_mesh_t m : handles)
            if (!m) return BCHAR_ERR_INVALID_ARG;
        std::sort(handles.begin(), handles.end());
        if (std::adjacent_find(handles.begin(), handles.end()) != handles.end())
            return BCHAR_ERR_INVALID_ARG;  // a handle may be stepped by one thread at a time

        std::vector<int> order(count);
        std::iota(order.begin(), order.end(), 0);
        std::stable_sort(order.begin(), order.end(),
                         [&](int a, int b) { return meshes[a]->nc > meshes[b]->nc; });
        std::vector<bchar_status> st(count, BCHAR_OK);
        std::atomic<int> next{0};
        auto work = [&]() {
            for (;;) {
                const int k = next.fetch_add(1);
                if (k >= count) break;
                const int i = order[k];
                bchar_mesh_t m = meshes[i];
                if (cudaSetDevice(m->device) != cudaSuccess) {
                    cudaGetLastError();
                    st[i] = BCHAR_ERR_CUDA;
                    continue;
                }
                st[i] = bchar_step(m, dt[i], c_in[i], c_out[i], c_dtype[i], infos ? &infos[i] : nullptr);
            }
        };
        int workers = max_workers > 0 ? max_workers : kDefaultWorkers;
        if (workers > count) workers = count;
        std::vector<std::thread> pool;
        try {
            for (int w = 1; w < workers; ++w) pool.emplace_back(work);
        } catch (const std::exception &) {
            // fewer threads than asked for: the ones running and this thread finish the batch
        }
        work();
        for (std::thread &t : pool) t.join();
        cudaSetDevice(caller_device);  // this thread stepped handles too
        bchar_status first = BCHAR_OK;
        for (int i = 0; i < count; ++i) {
            if (statuses) statuses[i] = st[i];
            if (first == BCHAR_OK && st[i] != BCHAR_OK) first = st[i];
        }
        return first;
    } catch (const std::exception &) {
        return BCHAR_ERR_OUT_OF_MEMORY;
    }
}
