"""CPU oracle of the VEG splatting path (test infrastructure only)."""
