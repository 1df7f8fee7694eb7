"""GB300-native LBM-RANS hot path (arXiv 2601.18443)."""
