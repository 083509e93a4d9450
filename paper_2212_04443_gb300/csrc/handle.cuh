// Handle state: stream, error text, grow-only device workspace.
#pragma once
#include <string>
#include <vector>

#include "common.cuh"
#include "kernels.cuh"

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  template <typename T>
  T* as() const {
    return reinterpret_cast<T*>(p);
  }
};

struct bchdav_handle_s {
  cudaStream_t stream = nullptr;
  bool owns_stream = false;   // created by the library (batched workers): destroyed with it
  // second stream and two events for work that runs beside the main stream (Step 9 accumulates
  // Q there); created on first use, ordered against `stream` by the events only
  cudaStream_t aux_stream = nullptr;
  cudaEvent_t aux_ev[2] = {nullptr, nullptr};
  bool ensure_aux_stream() {
    if (aux_stream) return true;
    if (cudaStreamCreateWithFlags(&aux_stream, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&aux_ev[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&aux_ev[1], cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      release_aux_stream();
      return false;
    }
    return true;
  }
  void release_aux_stream() {
    if (aux_stream) {
      cudaStreamSynchronize(aux_stream);
      cudaStreamDestroy(aux_stream);
    }
    for (cudaEvent_t& e : aux_ev) {
      if (e) cudaEventDestroy(e);
      e = nullptr;
    }
    aux_stream = nullptr;
  }
  int device = 0;
  // > 0: block cap of the cooperative kernels (1 for handles whose kernels may run beside
  // another handle's, so that no cooperative grid can be left partly resident)
  int coop_grid_cap = 0;
  int sms = bchdav::kSMs;
  std::string err;
  std::vector<DevBuf*> owned;
  // workspace slots
  DevBuf V, W, Vtmp, Xo, F[4], H, G, Y, D, part, eigw, small, norm0, val32, R;
  DevBuf hrow, hcol, hval, hvinit, hev, hevec;   // device copies for bchdav_solve_host
  DevBuf Rres, mix;   // mixed path: residual block of Step 12, per-column filter coefficients
  DevBuf oz;          // slices of the float64-accurate tensor-core products
  DevBuf oz_vt, oz_vr, oz_xt, oz_bw, oz_part;   // cached planes: V by columns, V by rows, X by columns
  DevBuf tc_err;                                // set by a tensor-core kernel whose wait expired
  // long-row schedule of the CSR matrix in use (rows over the segment threshold)
  DevBuf lg_cnt, lg_off, lg_tiles, lg_row, lg_pseg;
  bchdav::SpmmLong lg;
  DevBuf gnn, gnn_opt, gnn_w;   // start-block network: activations, optimiser state, Ritz step
  DevBuf km, km_x;              // clustering: centroids, sums, seeding state; transposed features
  DevBuf lz;                    // Lanczos bound estimate: three vectors, coefficients, T_k
  DevBuf vchk;                  // count of non-finite entries of a caller's V_init
  DevBuf vallo, ddx;            // mixed path: A's values' low float parts; split block scratch
  const bchdav::SpmmLong* long_rows() const { return lg.n_seg > 0 ? &lg : nullptr; }
  std::vector<bchdav_iter_record> history;
  // filter SpMM schedules found by timing (block size of the row kernel per matrix and width)
  struct SpmmTuneEntry {
    const int* rowptr;
    int n;
    long long nnz;
    int b, vsize, threads;
  };
  std::vector<SpmmTuneEntry> spmm_tune;
  // worker handles of bchdav_solve_batched (own streams, cooperative grids capped at one block)
  std::vector<bchdav_handle_s*> workers;
  int batch_workers = 8;
  // Pinned staging.  host_pinned belongs to the solve driver; host_aux to the
  // step helpers (filter coefficients, orthonormalisation scalars).  Each helper
  // synchronises the stream before it writes host_aux again, and nothing writes
  // host_pinned while a copy from it may still be queued.
  double* host_pinned = nullptr;
  size_t host_pinned_doubles = 0;
  double* host_aux = nullptr;
  size_t host_aux_doubles = 0;

  // Cap on the device workspace this handle may hold (bytes; 0 = no cap).  A request that
  // would exceed it fails with BCHDAV_ERR_OOM before anything is freed, as a failed
  // cudaMalloc does, so the handle stays usable.
  size_t mem_limit = 0;

  void set_error(bchdav_status, const std::string& m) { err = m; }

  bchdav_status ensure(DevBuf& b, size_t bytes) {
    if (bytes == 0) bytes = 16;
    if (b.bytes >= bytes) return BCHDAV_OK;
    if (mem_limit > 0 && held_bytes() - b.bytes + bytes > mem_limit) {
      err = std::string("device allocation of ") + std::to_string(bytes) +
            " bytes would exceed the handle's workspace limit of " + std::to_string(mem_limit) +
            " bytes";
      return BCHDAV_ERR_OOM;
    }
    b.release();
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
      cudaGetLastError();
      b.p = nullptr;
      err = std::string("device allocation of ") + std::to_string(bytes) + " bytes failed: " +
            cudaGetErrorString(e);
      return BCHDAV_ERR_OOM;
    }
    b.bytes = bytes;
    return BCHDAV_OK;
  }

  bchdav_status ensure_pinned(size_t doubles) {
    if (host_pinned_doubles >= doubles) return BCHDAV_OK;
    if (host_pinned) cudaFreeHost(host_pinned);
    host_pinned = nullptr;
    cudaError_t e = cudaMallocHost(&host_pinned, doubles * sizeof(double));
    if (e != cudaSuccess) {
      cudaGetLastError();
      err = "pinned host allocation failed";
      host_pinned_doubles = 0;
      return BCHDAV_ERR_OOM;
    }
    host_pinned_doubles = doubles;
    return BCHDAV_OK;
  }

  bchdav_status ensure_aux(size_t doubles) {
    if (host_aux_doubles >= doubles) return BCHDAV_OK;
    cudaStreamSynchronize(stream);
    if (host_aux) cudaFreeHost(host_aux);
    host_aux = nullptr;
    cudaError_t e = cudaMallocHost(&host_aux, doubles * sizeof(double));
    if (e != cudaSuccess) {
      cudaGetLastError();
      err = "pinned host allocation failed";
      host_aux_doubles = 0;
      return BCHDAV_ERR_OOM;
    }
    host_aux_doubles = doubles;
    return BCHDAV_OK;
  }

  // every workspace slot (for the accounting of mem_limit and for release_all)
  template <typename Fn>
  void for_each_buf(Fn f) {
    DevBuf* all[] = {&V, &W, &Vtmp, &Xo, &F[0], &F[1], &F[2], &F[3], &H, &G, &Y, &D, &part, &eigw,
                     &small, &norm0, &val32, &R, &hrow, &hcol, &hval, &hvinit, &hev, &hevec, &Rres,
                     &mix, &oz, &oz_vt, &oz_vr, &oz_xt, &oz_bw, &oz_part, &tc_err, &lg_cnt,
                     &lg_off, &lg_tiles, &lg_row, &lg_pseg, &gnn, &gnn_opt, &gnn_w, &km, &km_x,
                     &lz, &vchk, &vallo, &ddx};
    for (DevBuf* b : all) f(b);
  }
  size_t held_bytes() {
    size_t t = 0;
    for_each_buf([&](DevBuf* b) { t += b->bytes; });
    return t;
  }

  void release_all() {
    release_aux_stream();
    lg = bchdav::SpmmLong();
    for_each_buf([](DevBuf* b) { b->release(); });
    for (bchdav_handle_s* w : workers) {
      cudaStreamSynchronize(w->stream);
      w->release_all();
      if (w->owns_stream) cudaStreamDestroy(w->stream);
      delete w;
    }
    workers.clear();
    if (host_pinned) cudaFreeHost(host_pinned);
    host_pinned = nullptr;
    host_pinned_doubles = 0;
    if (host_aux) cudaFreeHost(host_aux);
    host_aux = nullptr;
    host_aux_doubles = 0;
  }
};

// Long-row schedule of A (rows with more than kLongRow nonzeros become segments) with segment
// workspace for products up to width_bytes per row (solver.cu); one host synchronisation.
bchdav_status prepare_long_rows(bchdav_handle h, const bchdav_csr* A, size_t width_bytes);

namespace bchdav {
// k-step Lanczos bound estimate of the spectrum of A (lanczos.cu): lowb = theta_min,
// upperb = theta_max + beta_k; alpha/beta (host, may be NULL) receive the coefficients of the
// steps done (fewer than `steps` when some beta_j is exactly 0).
bchdav_status lanczos_bounds(bchdav_handle h, const bchdav_csr* A, int steps,
                             unsigned long long seed, double* lowb, double* upperb,
                             double* alpha_out, double* beta_out, int* steps_done);
}  // namespace bchdav
