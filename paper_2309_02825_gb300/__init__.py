"""GB300-native Cole-Hopf fourth-order MRT-LB solver (arXiv:2309.02825)."""
