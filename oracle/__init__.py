"""FP64 CPU oracle: test infrastructure only (tests, smoke check, CPU baseline).

The CUDA library never imports this package; the two share no code."""
