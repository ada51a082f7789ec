"""GB300-native splatting core of Volume Encoding Gaussians (arXiv 2504.13339)."""
