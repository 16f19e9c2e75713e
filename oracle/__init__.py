"""FP64 CPU oracle of the two-beam FFT BPM (test infrastructure only)."""
