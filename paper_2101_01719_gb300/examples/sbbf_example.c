/*
 * The C ABI used from plain C99: build a filter from device-generated hashes,
 * look up members and fresh hashes, union two filters, hash raw keys on the
 * device, and round-trip the filter through the native serialized format.
 *
 * Build (from the repository root, after the library is built):
 *   gcc -std=c99 -O2 -Iinclude -I/usr/local/cuda/include \
 *       paper_2101_01719_gb300/examples/sbbf_example.c \
 *       -Lpaper_2101_01719_gb300 -lsbbf -L/usr/local/cuda/lib64 -lcudart \
 *       -Wl,-rpath,$PWD/paper_2101_01719_gb300 -o sbbf_example
 * Prints one line "members N/N fresh-hits F union-ok 1 keys-ok 1 serialize-ok 1"
 * and exits 0 when every check holds.
 */
#include <cuda_runtime.h>
#include <stdint.h>
#include <stdio.h>
#include <stdlib.h>

#include "sbbf.h"

#define CHECK(call)                                                        \
  do {                                                                     \
    sbbf_status st_ = (call);                                              \
    if (st_ != SBBF_OK) {                                                  \
      fprintf(stderr, "%s failed: %s\n", #call, sbbf_status_string(st_)); \
      return 1;                                                            \
    }                                                                      \
  } while (0)

static unsigned long long count_hits(const uint32_t *d_bits, size_t n) {
  unsigned long long *d_count = NULL, count = 0;
  if (cudaMalloc((void **)&d_count, sizeof(count)) != cudaSuccess) return ~0ull;
  if (sbbf_count_bits(d_bits, n, d_count, NULL) != SBBF_OK) return ~0ull;
  cudaMemcpy(&count, d_count, sizeof(count), cudaMemcpyDeviceToHost);
  cudaFree(d_count);
  return count;
}

int main(void) {
  const uint32_t num_blocks = 32768; /* 1 MiB */
  const size_t n = 1000000, q = 1 << 22;
  uint64_t *d_keys = NULL, *d_fresh = NULL;
  uint32_t *d_bits = NULL;
  if (cudaMalloc((void **)&d_keys, n * 8) != cudaSuccess ||
      cudaMalloc((void **)&d_fresh, q * 8) != cudaSuccess ||
      cudaMalloc((void **)&d_bits, ((q + 31) / 32) * 4) != cudaSuccess) {
    fprintf(stderr, "cudaMalloc failed\n");
    return 1;
  }
  CHECK(sbbf_fill_splitmix64(d_keys, n, 12345, 0, NULL));
  CHECK(sbbf_fill_splitmix64(d_fresh, q, 67890, 0, NULL));

  sbbf_t *f = NULL, *g = NULL, *h = NULL;
  CHECK(sbbf_create(num_blocks, &f));
  CHECK(sbbf_insert_hashes(f, d_keys, n, NULL));

  /* every inserted hash is found */
  CHECK(sbbf_find_hashes(f, d_keys, n, d_bits, NULL));
  const unsigned long long members = count_hits(d_bits, n);
  /* fresh hashes: the false-positive rate of 30.5 hashes per block (~2.7%) */
  CHECK(sbbf_find_hashes(f, d_fresh, q, d_bits, NULL));
  const unsigned long long fresh = count_hits(d_bits, q);
  const double fpr = (double)fresh / (double)q;

  /* union: g holds the first half, h the second; g | h answers for all */
  CHECK(sbbf_create(num_blocks, &g));
  CHECK(sbbf_create(num_blocks, &h));
  CHECK(sbbf_insert_hashes(g, d_keys, n / 2, NULL));
  CHECK(sbbf_insert_hashes(h, d_keys + n / 2, n - n / 2, NULL));
  CHECK(sbbf_union(g, h, NULL));
  uint32_t *w_f = (uint32_t *)malloc((size_t)num_blocks * 32);
  uint32_t *w_g = (uint32_t *)malloc((size_t)num_blocks * 32);
  CHECK(sbbf_copy_to_host(f, w_f, (size_t)num_blocks * 32, NULL));
  CHECK(sbbf_copy_to_host(g, w_g, (size_t)num_blocks * 32, NULL));
  int union_ok = 1;
  for (size_t i = 0; i < (size_t)num_blocks * 8; ++i) union_ok &= w_f[i] == w_g[i];

  /* raw keys hashed on the device: fused insert equals hash-then-insert */
  CHECK(sbbf_clear(g, NULL));
  CHECK(sbbf_clear(h, NULL));
  CHECK(sbbf_insert_keys(g, d_keys, 8, n, 0, NULL));
  CHECK(sbbf_hash_keys(d_keys, 8, n, 0, d_fresh, NULL));
  CHECK(sbbf_insert_hashes(h, d_fresh, n, NULL));
  uint32_t *w_h = (uint32_t *)malloc((size_t)num_blocks * 32);
  CHECK(sbbf_copy_to_host(g, w_g, (size_t)num_blocks * 32, NULL));
  CHECK(sbbf_copy_to_host(h, w_h, (size_t)num_blocks * 32, NULL));
  int keys_ok = 1;
  for (size_t i = 0; i < (size_t)num_blocks * 8; ++i) keys_ok &= w_g[i] == w_h[i];

  /* serialize and read back */
  const size_t bytes = sbbf_serialized_size(f);
  void *buf = malloc(bytes);
  sbbf_t *back = NULL;
  CHECK(sbbf_serialize(f, buf, bytes, NULL));
  CHECK(sbbf_deserialize(buf, bytes, &back));
  CHECK(sbbf_copy_to_host(back, w_h, (size_t)num_blocks * 32, NULL));
  int serialize_ok = sbbf_num_blocks(back) == num_blocks;
  for (size_t i = 0; i < (size_t)num_blocks * 8; ++i) serialize_ok &= w_f[i] == w_h[i];

  printf("members %llu/%zu fresh-hits %llu union-ok %d keys-ok %d serialize-ok %d\n", members,
         n, fresh, union_ok, keys_ok, serialize_ok);
  const int ok = members == n && fpr > 0.02 && fpr < 0.035 && union_ok && keys_ok && serialize_ok;

  free(buf);
  free(w_f);
  free(w_g);
  free(w_h);
  sbbf_destroy(back);
  sbbf_destroy(h);
  sbbf_destroy(g);
  sbbf_destroy(f);
  cudaFree(d_keys);
  cudaFree(d_fresh);
  cudaFree(d_bits);
  return ok ? 0 : 2;
}
