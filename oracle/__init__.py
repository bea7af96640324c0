"""CPU FP64 oracle: TEST INFRASTRUCTURE ONLY (tests, smoke(), the benchmark's CPU baseline)."""
