// Internal launch interface between the C ABI (dil_abi.cu) and the kernel
// translation units.  Not part of the public ABI.
#pragma once
#include <cstddef>
#include <cstdint>

#include <cuda_runtime.h>

namespace dil {

enum Op { OP_KEYGEN = 0, OP_SIGN = 1, OP_VERIFY = 2 };

// Scratch polynomials (256 int32 each) one task of `op` needs in the plain form.
size_t scratch_polys(int op, int level);
// Dynamic shared memory of a CTA with `warps` warps.
size_t cta_smem_bytes(int warps);

cudaError_t launch_keygen(int level, int n, const uint8_t *seeds, uint8_t *pk, uint8_t *sk, int32_t *scratch,
                          int warps, cudaStream_t s);
cudaError_t launch_sign(int level, int n, const uint8_t *sk, const uint8_t *msg, const uint64_t *off,
                        uint8_t *sig, int32_t *status, int32_t *iters, int32_t *scratch, int max_iter,
                        int warps, cudaStream_t s);
cudaError_t launch_verify(int level, int n, const uint8_t *pk, const uint8_t *msg, const uint64_t *off,
                          const uint8_t *sig, uint8_t *ok, int32_t *scratch, int warps, cudaStream_t s);

// primitives (test-only entry points)
cudaError_t launch_test_shake(int kind, int n, const uint8_t *in, const uint64_t *off, uint8_t *out,
                              int outlen, cudaStream_t s);
cudaError_t launch_test_ntt(int n, const int32_t *in, int32_t *out, int inverse, cudaStream_t s);
cudaError_t launch_test_expand_a(int level, int n, const uint8_t *rho, int32_t *out, cudaStream_t s);
cudaError_t launch_test_expand_s(int level, int n, const uint8_t *rhop, int32_t *out, cudaStream_t s);
cudaError_t launch_test_expand_mask(int level, int n, const uint8_t *rhop, const int32_t *kappa, int32_t *out,
                                    cudaStream_t s);
cudaError_t launch_test_sample_in_ball(int level, int n, const uint8_t *ct, int32_t *out, cudaStream_t s);
cudaError_t launch_test_rounding(int level, int n, const int32_t *r, const int32_t *z, const uint8_t *h,
                                 int32_t *out, cudaStream_t s);

// test-only issue-rate probe (thread-ops per SM clock)
cudaError_t measure_issue_rate(int op, double *rate);

}  // namespace dil
