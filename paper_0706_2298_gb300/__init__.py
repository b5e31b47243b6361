"""GB300-native deflated SAP-GCR solver for the Wilson-clover Dirac equation."""
