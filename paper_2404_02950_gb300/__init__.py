"""GB300-native AMR axion-string stepper (placeholder; binding added with the library)."""
