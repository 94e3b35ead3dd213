"""B300-native transport-based rendering (TBR) with capsule deposition strokes."""
