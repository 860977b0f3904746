// Chunked host<->device transfer-and-convert engine.
#pragma once

#include <cuda_runtime.h>

#include <mutex>
#include <vector>

#include "mrn_internal.h"

namespace mrn {

// One contiguous piece of a view's storage.
struct ViewPart {
  char* ptr;
  uint64_t bytes;
};

// The storage pieces of a view in a fixed order: AoS base (+ child pool);
// AoSoA base; SoA data columns (+ offsets, child columns).
std::vector<ViewPart> view_parts(const mrn_view& v);
// Records [r0, r0 + cnt) of a view of a non-jagged schema, as a view of its
// own.  SoA sub-views use per-column pointers stored in `cols`.  AoSoA
// sub-views need r0 to be a multiple of B.
mrn_view sub_view(const mrn_view& v, uint64_t r0, uint64_t cnt, std::vector<void*>& cols);
// A device view shaped like `like` (same schema, layout, sizes) with its
// parts packed at `stage` (stage == nullptr: size only).  Returns the bytes.
uint64_t staged_view(const mrn_view& like, char* stage, mrn_view* out, std::vector<void*>& cols,
                     std::vector<void*>& ccols);
// Bytes per record of a layout (AoSoA: block bytes / B, rounded up).
uint64_t record_bytes(const mrn_schema* s, const mrn_layout& l);

// Staging slots, copy/compute streams and events of one pipeline.  Not
// thread-safe by itself: callers serialise run() (the default engine of a
// device holds a mutex; the server gives each slot its own engine).
class TransferEngine {
 public:
  TransferEngine() = default;
  ~TransferEngine();
  TransferEngine(const TransferEngine&) = delete;
  TransferEngine& operator=(const TransferEngine&) = delete;

  // Device bytes this engine holds for the given options and request.
  static uint64_t staging_bytes(const mrn_view& src, const mrn_view& dst, uint64_t chunk_bytes,
                                int n_slots);
  // Runs one transfer-and-convert ordered after `user` and before later
  // work on `user`.  Device staging comes from `arena` when non-null
  // (arena_bytes long), else from the engine's own allocation.
  int run(const mrn_view& src, const mrn_view& dst, uint64_t chunk_bytes, int n_slots,
          cudaStream_t user, char* arena = nullptr, uint64_t arena_bytes = 0);
  // Stream on which the engine's last work completes.
  cudaStream_t done_stream() const { return s_conv_; }

 private:
  int init();
  int ensure_staging(uint64_t bytes);
  int ensure_whole(int h, uint64_t bytes);
  int run_whole(const mrn_view& src, const mrn_view& dst, cudaStream_t user, char* stage,
                uint64_t stage_bytes);
  int run_chunked(const mrn_view& src, const mrn_view& dst, uint64_t R, uint64_t stride, int n_slots, char* stage);

  bool ready_ = false;
  cudaStream_t s_copy_ = nullptr, s_conv_ = nullptr;
  std::vector<cudaEvent_t> ev_copied_, ev_free_;
  cudaEvent_t ev_start_ = nullptr, ev_copy_done_ = nullptr, ev_done_ = nullptr;
  char* staging_ = nullptr;
  uint64_t staging_bytes_ = 0;
  // The slots the last chunked call used (staging base, slot stride, slot
  // count) and the slot its successor takes first.  A chunked call with the
  // same slots waits only for each slot it reuses, so its first copies
  // overlap the previous call's last conversions; any other call waits for
  // the previous call to finish.
  const char* pipe_stage_ = nullptr;
  uint64_t pipe_stride_ = 0;
  int pipe_slots_ = 0;
  int next_slot_ = 0;
  // Calls that stage a whole source (jagged schemas) take two buffers of
  // their own in turn: a call waits only until the call before last has
  // finished with its buffer, so its copy overlaps the previous call's
  // conversion.
  char* whole_[2] = {};
  uint64_t whole_bytes_[2] = {};
  cudaEvent_t ev_whole_free_[2] = {};
  int next_whole_ = 0;
};

// Staging slot stride of chunked calls with `chunk_bytes` chunks: the same
// for every schema and layout pair whose chunk fits it (so that their calls
// can share slots), else the chunk's own size.
uint64_t slot_stride(uint64_t chunk_bytes, uint64_t slot_bytes);

}  // namespace mrn
