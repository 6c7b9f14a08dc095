// Host-side definitions shared by the C-ABI translation units (pb_api.cu,
// pb_batch.cu).  Not part of the public ABI.
#pragma once

#include <string>
#include <vector>

#include "pb_common.cuh"

struct pb_handle {
    int device = 0;
    int num_sms = 0;
    pb_alloc_fn alloc = nullptr;
    pb_free_fn free_fn = nullptr;
    void *ctx = nullptr;
    std::string last_error;
    cudaEvent_t phase_ev[4] = {nullptr, nullptr, nullptr, nullptr};
    bool phase_on = false;
    // batched products: tuned parameters per (log2 n, d class) sparsity class
    std::vector<pb_batch_tune> tuning;
    // pb_spgemm_host: streams for the bulk copies and for small reads (created on first use)
    cudaStream_t copy_stream = nullptr;
    cudaStream_t small_stream = nullptr;
    ~pb_handle() {
        if (copy_stream) cudaStreamDestroy(copy_stream);
        if (small_stream) cudaStreamDestroy(small_stream);
    }
};

namespace pb {

pb_status host_fail(pb_handle *h, pb_status st, const std::string &msg);
pb_status host_cuda_fail(pb_handle *h, cudaError_t e, const char *where);
pb_status host_check_operands(pb_handle *h, const pb_csc *A, const pb_csr *B);
// Device bytes a plan holds (its arena, work-item table and oversize map).
size_t plan_device_bytes(const pb_plan *p);

}  // namespace pb

#define PB_CUDA_H(h, call)                                                    \
    do {                                                                      \
        cudaError_t e_ = (call);                                              \
        if (e_ != cudaSuccess) return pb::host_cuda_fail((h), e_, #call);     \
    } while (0)
