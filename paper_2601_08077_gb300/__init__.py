"""GB300-native adaptive-precision density fitting (INT8-slice emulated DF K build)."""
