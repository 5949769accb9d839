"""FP64 reference implementation of HAP.  Test infrastructure only: the
product path never imports this package."""
