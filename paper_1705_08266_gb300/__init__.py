"""GB300-native 2-D DWT by non-separable lifting (Barina et al., arXiv 1705.08266)."""
