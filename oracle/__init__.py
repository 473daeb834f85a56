"""CPU oracle for the GPU file-read path.  TEST INFRASTRUCTURE ONLY.

Plain, slow, single-threaded restatement of what the GPU path computes, written
from the paper ("A readahead prefetcher for GPU file system layer", Dimitsas and
Silberstein) and nothing else.  It shares no code with the CUDA path; only the
seeded input generator in `inputs/` serves both.  Only `tests/`,
`__graft_entry__.smoke()` and `bench.py` (its CPU-baseline leg and
`--impl reference`) may import it; the product path never does.

Modules:
  plain   -- the plain definition of a gread (Section 2.2: a read returns the
             file's bytes) and of the per-stride checksums of the benchmark
             (Section 6.1 microbenchmark).  Exact integer arithmetic.
  policy  -- the page cache, readahead prefetcher and replacement policy
             (Sections 2.2, 2.3, 4.1, 5.1) stepped over a serialized gread
             trace, including the paper's own prefetcher with private
             buffers and its per-threadblock LRA replacement (also combined
             with this library's readahead); emits delivered bytes, the RPC
             log, the eviction log and counters.
  apps    -- the application-shaped consumers (Section 6.2 runs applications
             over GPUfs): float64 row dot products with the float32 error
             bound gamma_n, and exact integer histograms.

Parity status: `plain` is pinned by brute-force reads and by checksums
recomputed from the generator; `policy` is pinned by the worked readahead
example (Section 3.1), closed-form window sequences, fits-in-cache, streaming
and per-block-quota invariants, and hand-derived logs (tests/golden: a stream
through a 3-frame cache, the on-demand fallback, the paper's private buffer
with its LRA, readahead with the per-block LRA of two streams); `apps` is
pinned by math.fsum and closed forms (row dots) and brute-force counting
(histograms).  Policy *timing* under concurrency has several correct outcomes
and is only checked through invariants.
"""
