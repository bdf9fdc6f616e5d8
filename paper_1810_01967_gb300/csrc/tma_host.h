// Host helper shared by the tensor-core kernels: TMA descriptors of K-major operands.
#pragma once
#include <cuda.h>
#include "mrf_internal.cuh"

// Tensor map over a row-major [rows][Kp] operand of 2-byte (BF16) or 1-byte (E4M3) elements;
// boxes of 128 bytes (64 BF16 or 128 E4M3 elements) x box_rows rows with the 128-byte swizzle of
// the UMMA shared-memory descriptors.  The row pitch Kp x element size must be a multiple of 16
// bytes and the base 16-byte aligned; rows and columns beyond the tensor read as zero.
mrf_status tma_map_k128(CUtensorMap* m, const void* ptr, int64_t rows, int Kp, int box_rows,
                        bool f8);
