// fp_findpts_host: Find (and Interpolate) end to end from host memory, with
// the host<->device copies of some chunks of points overlapping the search
// of others.
//
// Every chunk's points go to the device on an upload stream, all issued up
// front; a compute stream (the caller's for even k, a second one for odd k)
// waits for chunk k's upload, searches the chunk (fp_findpts, with its cell
// order) and interpolates the field (fp_eval); a download stream waits for
// that and brings the chunk's results back.  Uploads and downloads run on
// separate streams so that they use both directions of the link at once and
// neither waits behind the other; only the first chunk's upload and the last
// chunk's download are not hidden behind kernels.  Two compute streams let
// the next chunk's persistent find launch take the SMs that the current one
// leaves during its tail (its last points run with few lanes), which a
// single stream would leave idle.
#include <stdlib.h>

#include <vector>

#include "fp_common.cuh"

namespace {

// Each chunk adds the tail of its find launch (a few tenths of a
// millisecond, partly hidden by the other compute stream) and hides the
// copies of all but the first upload and the last download (about 1.3 ms
// per 10^6 points in and out).  Measured on the 32^3 p=4 hex mesh with one
// field (find, eval and copies, L2 flushed before each call): at 10^6
// points two chunks are best, FP64 9.65 ms against 10.19 for one and 9.75,
// 9.89, 10.21 for three, four, five; FP_MIXED 3.76 against 3.87, 3.79,
// 3.87, 4.18; at 4x10^6 three or four were best (51.8 against 55.2 ms for
// one, an earlier FP64 kernel); so chunks of n/4 points, at least 2^19.
int64_t auto_chunk(int64_t n) {
  const int64_t c = (n + 3) / 4;
  return c < ((int64_t)1 << 19) ? ((int64_t)1 << 19) : c;
}

}  // namespace

extern "C" int fp_findpts_host(fp_mesh m, const double* pts_host, int64_t n, int32_t* code_host,
                               int32_t* elem_host, double* r_host, double* dist2_host,
                               const double* field_dev, int nc, double* out_host, int64_t chunk,
                               void* stream) {
  if (!m || n < 0 || n > INT32_MAX || chunk < 0) return FP_EINVAL;
  if (n == 0) return FP_OK;
  if (!pts_host || !code_host || !elem_host || !r_host || !dist2_host) return FP_EINVAL;
  if (field_dev && (nc <= 0 || !out_host)) return FP_EINVAL;
  if (!field_dev) nc = 0;
  const int d = m->d, dr = m->dr;
  const int64_t C = chunk > 0 ? (chunk < n ? chunk : n) : (auto_chunk(n) < n ? auto_chunk(n) : n);
  const int64_t K = (n + C - 1) / C;
  cudaStream_t st = (cudaStream_t)stream;
  // device buffers, in doubles: points, r, dist2, values; then code, elem
  const size_t nd = (size_t)n * (d + dr + 1) + (size_t)nc * n;
  const size_t bytes = nd * sizeof(double) + 2 * (size_t)n * sizeof(int32_t);
  char* buf = nullptr;
  if (cudaMallocAsync((void**)&buf, bytes, st) != cudaSuccess) return FP_ENOMEM;
  double* pts = (double*)buf;
  double* r = pts + (size_t)n * d;
  double* dist2 = r + (size_t)n * dr;
  double* out = dist2 + n;  // [K][nc][C]: each chunk's values together
  int32_t* code = (int32_t*)(out + (size_t)nc * n);
  int32_t* elem = code + n;
  cudaStream_t up = nullptr, down = nullptr, c1 = nullptr;
  // events: uploaded[k], computed[k], then the start and the three joins
  std::vector<cudaEvent_t> ev(2 * K + 4, nullptr);
  cudaEvent_t* uploaded = ev.data();
  cudaEvent_t* computed = ev.data() + K;
  cudaEvent_t& start = ev[2 * K];
  int rc = FP_OK;
  if (cudaStreamCreateWithFlags(&up, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&down, cudaStreamNonBlocking) != cudaSuccess ||
      cudaStreamCreateWithFlags(&c1, cudaStreamNonBlocking) != cudaSuccess)
    rc = FP_ELAUNCH;
  for (auto& e : ev)
    if (rc == FP_OK && cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) rc = FP_ELAUNCH;
  // FP_MIXED interpolation in double float: decided for the whole call (so
  // the values equal one fp_eval over all n points bit for bit) and the
  // field split once, before the chunks
  fp::DfField dff;
  const bool df = nc > 0 && fp::eval_uses_df(m, n);
  if (rc == FP_OK && df) rc = fp::df_field_prepare(m, field_dev, m->N, nc, &dff, st);
  // the other streams start after the allocation (and the split) on the caller's stream
  if (rc == FP_OK && (cudaEventRecord(start, st) != cudaSuccess || cudaStreamWaitEvent(up, start, 0) != cudaSuccess ||
                      cudaStreamWaitEvent(down, start, 0) != cudaSuccess ||
                      cudaStreamWaitEvent(c1, start, 0) != cudaSuccess))
    rc = FP_ELAUNCH;
  for (int64_t k = 0; k < K && rc == FP_OK; ++k) {
    const int64_t off = k * C, len = (n - off < C) ? n - off : C;
    if (cudaMemcpyAsync(pts + off * d, pts_host + off * d, sizeof(double) * len * d, cudaMemcpyHostToDevice,
                        up) != cudaSuccess ||
        cudaEventRecord(uploaded[k], up) != cudaSuccess)
      rc = FP_ELAUNCH;
  }
  for (int64_t k = 0; k < K && rc == FP_OK; ++k) {
    const int64_t off = k * C, len = (n - off < C) ? n - off : C;
    cudaStream_t cs = (k % 2 == 0) ? st : c1;
    if (cudaStreamWaitEvent(cs, uploaded[k], 0) != cudaSuccess) {
      rc = FP_ELAUNCH;
      break;
    }
    rc = fp_findpts(m, pts + off * d, len, code + off, elem + off, r + off * dr, dist2 + off, cs);
    double* o = out + (size_t)nc * off;
    if (rc == FP_OK && nc > 0)
      rc = df ? fp::df_field_eval(m, dff, code + off, elem + off, r + off * dr, len, o, cs)
              : fp_eval(m, code + off, elem + off, r + off * dr, len, field_dev, nc, o, cs);
    if (rc != FP_OK) break;
    if (cudaEventRecord(computed[k], cs) != cudaSuccess || cudaStreamWaitEvent(down, computed[k], 0) != cudaSuccess) {
      rc = FP_ELAUNCH;
      break;
    }
    cudaError_t e = cudaMemcpyAsync(code_host + off, code + off, sizeof(int32_t) * len, cudaMemcpyDeviceToHost, down);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(elem_host + off, elem + off, sizeof(int32_t) * len, cudaMemcpyDeviceToHost, down);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(r_host + off * dr, r + off * dr, sizeof(double) * len * dr, cudaMemcpyDeviceToHost, down);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(dist2_host + off, dist2 + off, sizeof(double) * len, cudaMemcpyDeviceToHost, down);
    if (e == cudaSuccess && nc > 0)  // [nc][len] on the device into rows of [nc][n]
      e = cudaMemcpy2DAsync(out_host + off, sizeof(double) * n, o, sizeof(double) * len, sizeof(double) * len, nc,
                            cudaMemcpyDeviceToHost, down);
    if (e != cudaSuccess) rc = FP_ELAUNCH;
  }
  // whatever happened, the buffer is freed after every copy and kernel
  if (c1 && cudaEventRecord(ev[2 * K + 1], c1) == cudaSuccess) cudaStreamWaitEvent(st, ev[2 * K + 1], 0);
  if (up && cudaEventRecord(ev[2 * K + 2], up) == cudaSuccess) cudaStreamWaitEvent(st, ev[2 * K + 2], 0);
  if (down && cudaEventRecord(ev[2 * K + 3], down) == cudaSuccess) cudaStreamWaitEvent(st, ev[2 * K + 3], 0);
  cudaFreeAsync(buf, st);
  fp::df_field_release(dff, st);
  const cudaError_t es = cudaStreamSynchronize(st);
  if (rc == FP_OK && es != cudaSuccess) rc = FP_ELAUNCH;
  for (auto& e : ev)
    if (e) cudaEventDestroy(e);
  if (up) cudaStreamDestroy(up);
  if (down) cudaStreamDestroy(down);
  if (c1) cudaStreamDestroy(c1);
  return rc;
}
