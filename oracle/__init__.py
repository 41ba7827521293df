"""Plain FP64 CPU oracle of the P3T soft step -- test infrastructure only."""
