"""FP64 CPU oracle of the GS-NFS per-frame codec (test infrastructure only)."""
