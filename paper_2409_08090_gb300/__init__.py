"""GB300-native nifty-ls hot path (placeholder; binding added with the CUDA library)."""
