"""GB300-native ensemble ODE solver (arXiv 2011.01740 method): Python binding."""
