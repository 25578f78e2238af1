"""Host logic of the batching form's autotuner (no GPU): the variants tried per grid."""
from paper_2205_06690_gb300 import batch
from paper_2205_06690_gb300 import binding as B


def test_variants_per_grid():
    big, small = 210e6, 26e6
    # register-pencil grids: pass kernels or persistent kernel, plain or streamed passes; chunks of
    # pairs only for the pass kernels and only where the batch exceeds one chunk
    v64 = batch._variants(64, B.SBSE_MIXED, big)
    assert (0, 1, 64) in v64 and (0, 1, 0) in v64 and (1, 1, 0) in v64
    assert all(c == 0 for p, t, c in v64 if p == 1)
    assert all(c == 0 for p, t, c in batch._variants(32, B.SBSE_MIXED, small))
    # the two-sweep grids have one kernel variant; only the chunking is tried
    assert batch._variants(96, B.SBSE_MIXED, 1e9) == [(0, 1, 0), (0, 1, 64)]
    # FP64: no streamed variants
    assert all(t == 1 for p, t, c in batch._variants(48, B.SBSE_FP64, big))
