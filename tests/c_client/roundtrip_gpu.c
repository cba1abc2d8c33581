/* A plain C99 client of the QTAM C ABI on the GPU, without PyTorch: reads
 * `batch` float32 segments of the 4 s workload from argv[1], runs
 * qtam_forward and qtam_inverse on device 0 with buffers from the CUDA
 * runtime's C API, and writes the complex64 envelopes to argv[2] and the
 * float32 reconstruction to argv[3].  Compiled and run by
 * tests/test_c_client.py (GPU part). */
#include <stdio.h>
#include <stdlib.h>

#include <cuda_runtime_api.h>

#include "qtam.h"

#define CHECK_CUDA(call)                                                              \
  do {                                                                                \
    cudaError_t e_ = (call);                                                          \
    if (e_ != cudaSuccess) {                                                          \
      fprintf(stderr, "%s: %s\n", #call, cudaGetErrorString(e_));                     \
      return 1;                                                                       \
    }                                                                                 \
  } while (0)
#define CHECK_QTAM(call)                                                              \
  do {                                                                                \
    qtam_status s_ = (call);                                                          \
    if (s_ != QTAM_OK) {                                                              \
      fprintf(stderr, "%s: %s: %s\n", #call, qtam_status_string(s_), qtam_last_error()); \
      return 1;                                                                       \
    }                                                                                 \
  } while (0)

static int read_all(const char* path, void* buf, size_t bytes) {
  FILE* f = fopen(path, "rb");
  size_t n;
  if (!f) return 1;
  n = fread(buf, 1, bytes, f);
  fclose(f);
  return n == bytes ? 0 : 1;
}
static int write_all(const char* path, const void* buf, size_t bytes) {
  FILE* f = fopen(path, "wb");
  size_t n;
  if (!f) return 1;
  n = fwrite(buf, 1, bytes, f);
  fclose(f);
  return n == bytes ? 0 : 1;
}

int main(int argc, char** argv) {
  static const double qs[] = {8.0, 16.0};
  const int64_t batch = 2;
  qtam_plan_desc d;
  qtam_plan_t plan = NULL;
  qtam_plan_info_t info;
  size_t ws_bytes = 0, x_bytes, y_bytes;
  float *hx, *hxh, *hy;
  void *dx, *dy, *dxh, *dws;

  if (argc != 4) {
    fprintf(stderr, "usage: %s x.bin y.bin xh.bin\n", argv[0]);
    return 2;
  }
  qtam_plan_desc_init(&d);
  d.sample_rate = 4096.0;
  d.length = 16384;
  d.q = qs;
  d.n_q = 2;
  d.f_min = 20.0;
  d.f_max = 1024.0;
  d.rows_per_plane = 32;
  CHECK_QTAM(qtam_plan(&d, 0, &plan));
  CHECK_QTAM(qtam_plan_info(plan, &info));
  CHECK_QTAM(qtam_workspace_size(plan, batch, &ws_bytes));
  x_bytes = (size_t)batch * (size_t)info.length * sizeof(float);
  y_bytes = (size_t)batch * (size_t)info.envelope_bytes_per_segment;

  hx = (float*)malloc(x_bytes);
  hxh = (float*)malloc(x_bytes);
  hy = (float*)malloc(y_bytes);
  if (!hx || !hxh || !hy || read_all(argv[1], hx, x_bytes)) {
    fprintf(stderr, "cannot read %s\n", argv[1]);
    return 1;
  }
  CHECK_CUDA(cudaMalloc(&dx, x_bytes));
  CHECK_CUDA(cudaMalloc(&dy, y_bytes));
  CHECK_CUDA(cudaMalloc(&dxh, x_bytes));
  CHECK_CUDA(cudaMalloc(&dws, ws_bytes));
  CHECK_CUDA(cudaMemcpy(dx, hx, x_bytes, cudaMemcpyHostToDevice));
  CHECK_QTAM(qtam_forward(plan, dx, batch, dy, dws, ws_bytes, NULL));
  CHECK_QTAM(qtam_inverse(plan, dy, batch, 0, dxh, dws, ws_bytes, NULL));
  CHECK_CUDA(cudaDeviceSynchronize());
  CHECK_CUDA(cudaMemcpy(hy, dy, y_bytes, cudaMemcpyDeviceToHost));
  CHECK_CUDA(cudaMemcpy(hxh, dxh, x_bytes, cudaMemcpyDeviceToHost));
  if (write_all(argv[2], hy, y_bytes) || write_all(argv[3], hxh, x_bytes)) {
    fprintf(stderr, "cannot write the outputs\n");
    return 1;
  }
  printf("M %d P %d K %d tau %.17g\n", (int)info.n_out, (int)info.n_planes, (int)info.rows_per_plane,
         info.p_floor_rel);
  CHECK_QTAM(qtam_destroy(plan));
  CHECK_CUDA(cudaFree(dx));
  CHECK_CUDA(cudaFree(dy));
  CHECK_CUDA(cudaFree(dxh));
  CHECK_CUDA(cudaFree(dws));
  free(hx);
  free(hxh);
  free(hy);
  return 0;
}
