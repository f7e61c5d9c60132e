"""B300-native batched nonlinear constraint projection (SNAP-FM hot path)."""
