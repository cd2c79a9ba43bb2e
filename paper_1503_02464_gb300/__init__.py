"""GB300-native relativistic particle-in-cell hot path (PICCANTE-style cycle)."""
