"""B300-native regularized minSR step for autoregressive GRU wave functions."""
