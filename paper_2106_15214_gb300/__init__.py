"""GB300-native joint-MM beta-NMF (see include/nmf.h for the C ABI)."""
