// Tensor-core first layer of the warm-start encoder (gmf_mlp_tc.cu).
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

// n_h1 must be a multiple of 16 in [16, 256].
int gmf_mlp_tc_check(int n_in, int n_h1, std::string* err);
// Elements of the BF16 copy of W1: n_h1 rows of n_in rounded up to 64 (zero padding).
size_t gmf_mlp_tc_w1_elems(int n_h1, int n_in);
// W1 (FP32, n_h1 x n_in) -> its padded BF16 copy, round to nearest even. Asynchronous.
int gmf_mlp_tc_weights(const float* W1, int n_h1, int n_in, __nv_bfloat16* W1b, cudaStream_t st);
// z1 = W1 log(1 + y) + b1 and h1 = gelu(z1) for `rows` cells (Z1 may be null). Asynchronous.
int gmf_mlp_tc_layer1(const void* Y, int y16, int64_t rows, int n_in, int n_h1, const __nv_bfloat16* W1b,
                      const float* b1, float* Z1, float* H1, unsigned* err_word, cudaStream_t st, std::string* err);
