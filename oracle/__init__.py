"""FP64 CPU oracle of the auxiliary-grid AMG method. Test infrastructure only."""
