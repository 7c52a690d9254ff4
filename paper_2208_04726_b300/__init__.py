"""B300-native differentiable Gauss-Newton bundle adjustment over the DPVO patch graph."""
